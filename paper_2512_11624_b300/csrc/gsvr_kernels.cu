// gsvr_kernels.cu -- the compute path of libgsvr.so (sm_103a).
//
// Per forward:
//   gauss_prep   Sigma_j = R(q) diag(exp(2 ls)) R(q)^T            (Sec. 2.2)
//   pose_prep    R_i = Rod(r) R0_i, t_i = Rod(r) c0_i + tau          (Sec. 2.4)
//   rec_count / rec_emit
//                every (slice i, Gaussian j): m = R_i^T (mu_j - t_i),
//                K = R_i^T Sigma_j R_i + Sigma_PSF (= R_i^T Sigma_obs R_i, Eq. 4);
//                keep if m_z^2 / K_zz <= r_c^2 (Mahalanobis cut); the pair's
//                restriction to the slice plane is the exact 2D Gaussian
//                w exp(-1/2 (u - c)^T P2 (u - c)) with P2 = Schur complement
//                inverse, c = m_xy - K_xz m_z / K_zz,
//                w = c_j sqrt(det Sigma_j / det K) exp(-1/2 m_z^2 / K_zz)  (Eq. 5 numerator)
//   key_emit     one key per (non-empty tile, record) in the record's bounding box
//   radix sort   keys by tile id (stable: within a tile records stay in Gaussian order)
//   gather       tile-ordered copy of the records
//   forward      per tile: records staged through shared memory by the TMA bulk
//                engine (double-buffered, mbarrier-completed), thread per pixel,
//                fused residual and loss
// Per backward:
//   backward     per tile: thread per record, pixels broadcast from shared
//                memory; 6 first/second moments of r_bar * e per (tile, record)
//   gauss_grad   thread per Gaussian: sums its records' moments, chains them to
//                mu, Sigma_j -> (ls, q), c; slice-frame gradients reduced in
//                shared memory, then one float64 atomic per (block, slice, entry)
//   pose_grad    (R_i, t_i) gradients -> (r, tau) through the exponential map
//   adam         fused, per-group learning rates
#include <math.h>

#include <cmath>

#include <algorithm>
#include <atomic>

#include "gsvr_launch.cuh"

namespace gsvr {

namespace {

constexpr float kNegHalfLog2e = -0.72134752044448170368f;  // -1/2 log2(e)

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void rodrigues_d(const double r[3], double R[9]) {
    const double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double th = sqrt(th2);
    double A, B;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0.0, -r[2], r[1], r[2], 0.0, -r[0], -r[1], r[0], 0.0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double k2 = K[3 * a] * K[b] + K[3 * a + 1] * K[3 + b] + K[3 * a + 2] * K[6 + b];
            R[3 * a + b] = (a == b ? 1.0 : 0.0) + A * K[3 * a + b] + B * k2;
        }
}

// Double-single arithmetic (a value carried as an unevaluated float32 sum
// hi + lo): TwoSum (Knuth) and the FMA-based exact product.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// u . x - o with u, o given as (hi, lo) pairs and x exact float32; result to
// ~2^-44 relative of the terms, returned rounded to float32 (hi) plus remainder (lo).
__device__ __forceinline__ float ds_dot_sub(const float uh[3], const float ul[3], const float x[3], float oh,
                                            float ol, float &lo) {
    const float p0 = __fmul_rn(uh[0], x[0]), p1 = __fmul_rn(uh[1], x[1]), p2 = __fmul_rn(uh[2], x[2]);
    const float e0 = fmaf(uh[0], x[0], -p0), e1 = fmaf(uh[1], x[1], -p1), e2 = fmaf(uh[2], x[2], -p2);
    float s, t1, t2, t3;
    two_sum(p0, p1, s, t1);
    two_sum(s, p2, s, t2);
    two_sum(s, -oh, s, t3);
    const float small = ((e0 + e1) + e2) + ((t1 + t2) + t3) + (ul[0] * x[0] + ul[1] * x[1] + ul[2] * x[2]) - ol;
    float hi;
    two_sum(s, small, hi, lo);
    return hi;
}

// Everything the record and its gradient need about one (slice, Gaussian) pair
// (float32; the mean's slice coordinates in double-single).
struct RecGeom {
    float R[9];       // slice rotation
    float d[3];       // mu - t (world)
    float mz;         // slice-normal coordinate of the mean
    float Kxx, Kyy, Kzz, Kxy, Kxz, Kyz;
    float qz;         // m_z^2 / K_zz
    float M2xx, M2yy, M2xy, det2;
    float P2xx, P2yy, P2xy;
    float w0;         // w / c_j
    float cb, ca;     // conditional centre, slice-centred pixel units (centre pass only)
};

// Cheap float32 rejection before the exact test: |m_z| against the cut with a
// relative margin (the exact test follows in rec_geom).
__device__ __forceinline__ bool slab_candidate(const float4 g0, const float4 g1, const float mu[3],
                                               const SliceDev &S, float rc2) {
    const float nx = S.nz_h[0], ny = S.nz_h[1], nz = S.nz_h[2];
    const float mz = nx * mu[0] + ny * mu[1] + nz * mu[2] - S.oz_h;
    const float sx = g0.x * nx + g0.w * ny + g1.x * nz;
    const float sy = g0.w * nx + g0.y * ny + g1.y * nz;
    const float sz = g1.x * nx + g1.y * ny + g0.z * nz;
    const float kzz = nx * sx + ny * sy + nz * sz + S.var[2];
    return mz * mz <= (rc2 * 1.001f + 1e-3f) * kzz + 1e-3f;
}

// The slice-frame fields the gradient's record geometry reads (rec_geom
// without the centre), staged in shared memory by the gradient epilogue; the
// field names follow SliceDev, so rec_geom<false> takes either.
struct SliceGeo {
    float R[9], t[3];
    float nz_h[3], nz_l[3];
    float oz_h, oz_l;
    float var[3];
    float dx, dy;
};
constexpr int kSliceGeoWords = (int)(sizeof(SliceGeo) / 4);  // 25
// Word offsets in SliceDev of the SliceGeo fields, in SliceGeo order.
__device__ __forceinline__ int slice_geo_src(int e) {
    return e < 12 ? e : (e < 18 ? e + 12 : e + 16);  // R, t | nz_h, nz_l | oz_h, oz_l, var, dx, dy
}
static_assert(offsetof(SliceDev, nz_h) == 24 * 4 && offsetof(SliceDev, oz_h) == 34 * 4 &&
                  offsetof(SliceDev, var) == 36 * 4 && offsetof(SliceDev, dy) == 40 * 4,
              "SliceGeo staging assumes the SliceDev layout");

template <bool CENTRE, typename SL>
__device__ __forceinline__ bool rec_geom(const float4 g0, const float4 g1, const float mu[3], const SL &S,
                                         float rc2, int norm_mode, RecGeom &G) {
    float zlo;
    const float zhi = ds_dot_sub(S.nz_h, S.nz_l, mu, S.oz_h, S.oz_l, zlo);
    G.mz = zhi + zlo;
    for (int e = 0; e < 9; ++e) G.R[e] = S.R[e];
    for (int a = 0; a < 3; ++a) G.d[a] = mu[a] - S.t[a];
    const float Sg[9] = {g0.x, g0.w, g1.x, g0.w, g0.y, g1.y, g1.x, g1.y, g0.z};
    float T[9];  // Sigma R
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            T[3 * a + b] = Sg[3 * a] * G.R[b] + Sg[3 * a + 1] * G.R[3 + b] + Sg[3 * a + 2] * G.R[6 + b];
    auto K = [&](int a, int b) { return G.R[a] * T[b] + G.R[3 + a] * T[3 + b] + G.R[6 + a] * T[6 + b]; };
    G.Kxx = K(0, 0) + S.var[0];
    G.Kyy = K(1, 1) + S.var[1];
    G.Kzz = K(2, 2) + S.var[2];
    G.Kxy = K(0, 1);
    G.Kxz = K(0, 2);
    G.Kyz = K(1, 2);
    G.qz = G.mz * G.mz / G.Kzz;
    if (!(G.qz <= rc2)) return false;
    const float ik = 1.0f / G.Kzz;
    G.M2xx = G.Kxx - G.Kxz * G.Kxz * ik;
    G.M2yy = G.Kyy - G.Kyz * G.Kyz * ik;
    G.M2xy = G.Kxy - G.Kxz * G.Kyz * ik;
    G.det2 = G.M2xx * G.M2yy - G.M2xy * G.M2xy;
    const float idet = 1.0f / G.det2;
    G.P2xx = G.M2yy * idet;
    G.P2yy = G.M2xx * idet;
    G.P2xy = -G.M2xy * idet;
    if (norm_mode == GSVR_NORM_EXACT)
        G.w0 = expf(g1.z - 0.5f * G.qz) * rsqrtf(G.Kzz * G.det2);
    else
        G.w0 = expf(-0.5f * G.qz);
    if constexpr (CENTRE) {
        // centre = m_xy - K_xz,yz m_z / K_zz, in pixels: (u . mu - o) - (K_xz / K_zz) m_z / dx
        float xlo, ylo;
        const float xhi = ds_dot_sub(S.ux_h, S.ux_l, mu, S.ox_h, S.ox_l, xlo);
        const float yhi = ds_dot_sub(S.uy_h, S.uy_l, mu, S.oy_h, S.oy_l, ylo);
        G.cb = (xhi - G.Kxz * ik * G.mz / S.dx) + xlo;
        G.ca = (yhi - G.Kyz * ik * G.mz / S.dy) + ylo;
    }
    return true;
}

// Tile bounding box of the record's ellipse {q <= r_c^2} on the slice.
__device__ __forceinline__ bool rec_bbox(const RecGeom &G, const SliceDev &S, float rc2, int tw, int th, int &tx0,
                                         int &tx1, int &ty0, int &ty1) {
    const float rho2 = fmaxf(rc2 - G.qz, 0.0f);
    const float hx = sqrtf(rho2 * G.M2xx) / S.dx;
    const float hy = sqrtf(rho2 * G.M2yy) / S.dy;
    const float blo = fminf(fmaxf(G.cb + S.cx0 - hx, -1.0f), (float)S.W);
    const float bhi = fminf(fmaxf(G.cb + S.cx0 + hx, -1.0f), (float)S.W);
    const float alo = fminf(fmaxf(G.ca + S.cy0 - hy, -1.0f), (float)S.H);
    const float ahi = fminf(fmaxf(G.ca + S.cy0 + hy, -1.0f), (float)S.H);
    const int b0 = max(0, (int)ceilf(blo)), b1 = min(S.W - 1, (int)floorf(bhi));
    const int a0 = max(0, (int)ceilf(alo)), a1 = min(S.H - 1, (int)floorf(ahi));
    if (!(G.det2 > 0.0f) || b0 > b1 || a0 > a1) return false;
    tx0 = b0 / tw;
    tx1 = b1 / tw;
    ty0 = a0 / th;
    ty1 = a1 / th;
    return true;
}

// Largest value over a rectangle of pixel centres [x0, x1] x [y0, y1] (slice-
// centred pixel units) of the record's exponent q(db, da) + log2 normal weight
// (log2 units; q is concave, so the maximum sits at the centre when it lies
// inside, else on an edge at the clamped stationary point).  The record's pair
// factors inside the rectangle are at most 2^(this).  Explicit roundings keep
// the result identical wherever it is evaluated.
// iAB = (-1/2 / A, -1/2 / B) of the record (rec_inv_ab), taken once per record.
__device__ __forceinline__ float2 rec_inv_ab(const Rec &R) {
    return make_float2(__fdiv_rn(-0.5f, R.a.z), __fdiv_rn(-0.5f, R.b.x));
}
__device__ __forceinline__ float rect_max_exponent(const Rec &R, float2 iAB, float x0, float x1, float y0, float y1) {
    const float A = R.a.z, C = R.a.w, B = R.b.x;
    const float X0 = __fsub_rn(x0, R.a.x), X1 = __fsub_rn(x1, R.a.x);
    const float Y0 = __fsub_rn(y0, R.a.y), Y1 = __fsub_rn(y1, R.a.y);
    if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return R.b.z;
    auto f = [&](float u, float v) {
        return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A, u), u), __fmul_rn(__fmul_rn(C, u), v)),
                         __fmul_rn(__fmul_rn(B, v), v));
    };
    const float iA = iAB.x, iB = iAB.y;
    float best = -INFINITY;
    const float Xs[2] = {X0, X1}, Ys[2] = {Y0, Y1};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float v = fminf(fmaxf(__fmul_rn(__fmul_rn(C, Xs[k]), iB), Y0), Y1);
        best = fmaxf(best, f(Xs[k], v));
        const float u = fminf(fmaxf(__fmul_rn(__fmul_rn(C, Ys[k]), iA), X0), X1);
        best = fmaxf(best, f(u, Ys[k]));
    }
    return __fadd_rn(best, R.b.z);
}

// Whether tile (tx, ty) of slice S has sampled pixels and the record reaches it.
__device__ __forceinline__ bool tile_live(const Rec &R, float2 iAB, const SliceDev &S, int tx, int ty, int tw, int th,
                                          const int *tps, const int *tpe, float qcut) {
    const int t = S.tile_base + ty * S.tiles_x + tx;
    if (tpe[t] <= tps[t]) return false;
    const float x0 = (float)(tx * tw) - S.cx0, x1 = (float)min(tx * tw + tw - 1, S.W - 1) - S.cx0;
    const float y0 = (float)(ty * th) - S.cy0, y1 = (float)min(ty * th + th - 1, S.H - 1) - S.cy0;
    return rect_max_exponent(R, iAB, x0, x1, y0, y1) >= qcut;
}

// Live tiles of a record's box; mask gets their row-major bits when the box
// has at most 32 tiles (else 0).
__device__ __forceinline__ int count_live_tiles(const Rec &R, const SliceDev &S, int tx0, int tx1, int ty0, int ty1,
                                                int tw, int th, const int *tps, const int *tpe, float qcut,
                                                unsigned &mask) {
    int n = 0, b = 0;
    const bool fits = (tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 32;
    const float2 iAB = rec_inv_ab(R);
    mask = 0u;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx, ++b)
            if (tile_live(R, iAB, S, tx, ty, tw, th, tps, tpe, qcut)) {
                ++n;
                if (fits) mask |= 1u << b;
            }
    return n;
}

// ------------------------------------------------------------- preprocessing
__global__ void k_gauss_prep(const float *__restrict__ th, int N, float4 *__restrict__ gpre, unsigned *status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float p[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) p[k] = th[(size_t)k * N + j];
    bool fin = true;
#pragma unroll
    for (int k = 0; k < 11; ++k) fin = fin && isfinite(p[k]);
    const float qn2 = p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9];
    if (!fin || !(qn2 > 0.0f)) atomicOr(status, ST_NONFINITE);
    const float iq = rsqrtf(qn2);
    float R[9];
    quat_rot(p[6] * iq, p[7] * iq, p[8] * iq, p[9] * iq, R);
    const float s0 = expf(2.f * p[3]), s1 = expf(2.f * p[4]), s2 = expf(2.f * p[5]);
    auto S = [&](int a, int b) { return R[3 * a] * s0 * R[3 * b] + R[3 * a + 1] * s1 * R[3 * b + 1] + R[3 * a + 2] * s2 * R[3 * b + 2]; };
    gpre[2 * j] = make_float4(S(0, 0), S(1, 1), S(2, 2), S(0, 1));
    gpre[2 * j + 1] = make_float4(S(0, 2), S(1, 2), p[3] + p[4] + p[5], p[10]);
}

__device__ __forceinline__ void split_pair(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

__global__ void k_pose_prep(const float *__restrict__ pose, const SliceStatic *__restrict__ ss,
                            SliceDev *__restrict__ sd, int M, unsigned *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double r[3], tau[3];
    bool fin = true;
    for (int k = 0; k < 3; ++k) {
        r[k] = pose[6 * i + k];
        tau[k] = pose[6 * i + 3 + k];
        fin = fin && isfinite(r[k]) && isfinite(tau[k]);
    }
    if (!fin) atomicOr(status, ST_NONFINITE);
    double Q[9], R[9], t[3];
    rodrigues_d(r, Q);
    const SliceStatic s = ss[i];
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b)
            R[3 * a + b] = Q[3 * a] * s.R0[b] + Q[3 * a + 1] * s.R0[3 + b] + Q[3 * a + 2] * s.R0[6 + b];
        t[a] = Q[3 * a] * s.c0[0] + Q[3 * a + 1] * s.c0[1] + Q[3 * a + 2] * s.c0[2] + tau[a];
    }
    SliceDev &o = sd[i];
    const double dx = o.dx, dy = o.dy;
    for (int e = 0; e < 9; ++e) o.R[e] = (float)R[e];
    for (int a = 0; a < 3; ++a) {
        o.t[a] = (float)t[a];
        split_pair(R[3 * a] / dx, o.ux_h[a], o.ux_l[a]);
        split_pair(R[3 * a + 1] / dy, o.uy_h[a], o.uy_l[a]);
        split_pair(R[3 * a + 2], o.nz_h[a], o.nz_l[a]);
    }
    split_pair((R[0] * t[0] + R[3] * t[1] + R[6] * t[2]) / dx, o.ox_h, o.ox_l);
    split_pair((R[1] * t[0] + R[4] * t[1] + R[7] * t[2]) / dy, o.oy_h, o.oy_l);
    split_pair(R[2] * t[0] + R[5] * t[1] + R[8] * t[2], o.oz_h, o.oz_l);
}

// ---------------------------------------------------------------- sampling
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long ctr) {
    unsigned long long z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Output t of the concatenated per-subject samples: subject k by binary search
// in out_first, then the keyed 4-round bijection on k bits with cycle walking
// (SplitMix64 round keys from seed + k * golden gamma and counter 4 step + r).
__global__ void k_sample_flags(int n_subj, const int *__restrict__ mask_first, const int *__restrict__ out_first,
                               int n_out, unsigned long long seed, unsigned long long step,
                               const unsigned long long *d_step, const int *__restrict__ mask_tpos,
                               int *__restrict__ flags) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_out) return;
    int lo = 0, hi = n_subj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (out_first[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int sj = lo;
    const int n_mask = mask_first[sj + 1] - mask_first[sj];
    if (n_mask <= 0) return;
    const unsigned long long stp = d_step ? *d_step : step;
    const unsigned long long sseed = seed + (unsigned long long)sj * 0x9E3779B97F4A7C15ull;
    int k = 1;
    while ((1ll << k) < (long long)n_mask) ++k;
    const int h = (k + 1) / 2;
    const unsigned long long msk = (k >= 64) ? ~0ull : ((1ull << k) - 1ull);
    unsigned long long xk[4], mul[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const unsigned long long key = splitmix64_at(sseed, 4ull * stp + (unsigned long long)r);
        xk[r] = key & msk;
        mul[r] = (key >> 32) | 1ull;
    }
    unsigned long long x = (unsigned long long)(t - out_first[sj]);
    // cycle walking terminates within 2^k steps (the rounds permute [0, 2^k))
    for (unsigned long long it = 0; it <= msk; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            x = (x ^ xk[r]) & msk;
            x = (x * mul[r]) & msk;
            x ^= x >> h;
        }
        if (x < (unsigned long long)n_mask) break;
    }
    if (x < (unsigned long long)n_mask) {
        const int m = mask_first[sj] + (int)x;  // rank among the masked pixels in tile order
        flags[mask_tpos ? mask_tpos[m] : m] = 1;
    }
}

__global__ void k_flags_from_list(const int *__restrict__ idx, int n, int n_pix, const uint8_t *__restrict__ mask,
                                  const int *__restrict__ pix_tpos, int *__restrict__ flags, unsigned *status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int p = idx[k];
    if (p < 0 || p >= n_pix) {
        atomicOr(status, ST_INDEX);
        return;
    }
    if (mask[p]) flags[pix_tpos[p]] = 1;
}

// List sample in masked-rank space: pix_mrank[p] = rank of pixel p among the
// masked pixels in tile order (-1 outside the mask).
__global__ void k_flags_from_list_rank(const int *__restrict__ idx, int n, int n_pix,
                                       const int *__restrict__ pix_mrank, int *__restrict__ flags,
                                       unsigned *status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int p = idx[k];
    if (p < 0 || p >= n_pix) {
        atomicOr(status, ST_INDEX);
        return;
    }
    const int m = pix_mrank[p];
    if (m >= 0) flags[m] = 1;
}

__global__ void k_compact(const int *__restrict__ flags, const int *__restrict__ pos,
                          const int *__restrict__ tile_sorted_pix, int n_pix, int *__restrict__ sampled) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pix) return;
    if (flags[t]) sampled[pos[t]] = tile_sorted_pix[t];
}

__global__ void k_tile_px_ranges(const int *__restrict__ sampled, const int *n_sampled, int cap,
                                 const int *__restrict__ pix_tile, int *start, int *end) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = min(*n_sampled, cap);
    if (s >= n) return;
    const int t = pix_tile[sampled[s]];
    if (s == 0 || pix_tile[sampled[s - 1]] != t) start[t] = s;
    if (s == n - 1 || pix_tile[sampled[s + 1]] != t) end[t] = s + 1;
}

__global__ void k_set_count(int *dst, int v) { *dst = v; }

// ------------------------------------------------------------------ binning
constexpr int kSliceChunk = 32;  // slices staged per round (one 32-bit candidate-mask word)

// Candidates: every (slice, Gaussian) pair whose slice-normal offset passes a
// float32 slab test with a small margin (a superset of the pairs the exact cut
// keeps).  Thread per Gaussian, slices staged through shared memory; the count
// pass sizes the Gaussian-major candidate list, the emit pass writes it.
template <bool EMIT>
__global__ void __launch_bounds__(128) k_cand(BinArgs a) {
    __shared__ SliceDev ssl[kSliceChunk];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < a.N;
    float mu[3] = {0.f, 0.f, 0.f};
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
    if (live) {
        mu[0] = a.theta[j];
        mu[1] = a.theta[a.N + j];
        mu[2] = a.theta[2 * a.N + j];
        g0 = a.gpre[2 * j];
        g1 = a.gpre[2 * j + 1];
    }
    int n = 0;
    const int base = EMIT && live ? a.rec_off[j] : 0;
    const int room = EMIT && live ? a.rec_off[j + 1] - base : 0;
    // a Gaussian meets only its own subject's slices; the block walks the union
    // of its threads' slice ranges (Gaussians of a subject are contiguous)
    int sl0 = 0, sl1 = a.M;
    if (a.gauss_subject) {
        __shared__ int blo, bhi;
        if (threadIdx.x == 0) {
            blo = a.M;
            bhi = 0;
        }
        __syncthreads();
        const bool on = live && (!a.subj_active || a.subj_active[a.gauss_subject[j]]);
        if (on) {
            const int sj = a.gauss_subject[j];
            sl0 = a.subj_slice_first[sj];
            sl1 = a.subj_slice_first[sj + 1];
            atomicMin(&blo, sl0);
            atomicMax(&bhi, sl1);
        }
        __syncthreads();
        if (!on) {  // (a retired subject's Gaussians meet no slice: no records, no work)
            sl0 = blo;
            sl1 = blo;
        }
        const int b0 = blo, b1 = bhi;
        __syncthreads();
        for (int i0 = b0; i0 < b1; i0 += kSliceChunk) {
            __syncthreads();
            const int nc = min(kSliceChunk, b1 - i0);
            {
                const int words = nc * (int)(sizeof(SliceDev) / 4);
                const int *src = reinterpret_cast<const int *>(a.slices + i0);
                int *dst = reinterpret_cast<int *>(ssl);
                for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
            }
            __syncthreads();
            if (!live) continue;
            for (int ii = 0; ii < nc; ++ii) {
                const int i = i0 + ii;
                if (i < sl0 || i >= sl1 || !slab_candidate(g0, g1, mu, ssl[ii], a.rc2)) continue;
                if (EMIT && n < room) {
                    const int c = base + n;
                    if (c < a.cap_rec) a.cand[c] = make_int2(j, i);
                    else atomicOr(a.status, ST_CAPACITY);
                }
                ++n;
            }
        }
        if (!EMIT && live) a.rec_cnt[j] = n;
        if (EMIT && live)
            for (int k = n; k < room && base + k < a.cap_rec; ++k) a.cand[base + k] = make_int2(j, -1);
        return;
    }
    for (int i0 = 0; i0 < a.M; i0 += kSliceChunk) {
        __syncthreads();
        const int nc = min(kSliceChunk, a.M - i0);
        {
            const int words = nc * (int)(sizeof(SliceDev) / 4);
            const int *src = reinterpret_cast<const int *>(a.slices + i0);
            int *dst = reinterpret_cast<int *>(ssl);
            for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        if (!live) continue;
        unsigned bits = 0u;  // (kSliceChunk = 32: chunk i0 / 32 is one mask word)
        for (int ii = 0; ii < nc; ++ii) {
            if (!slab_candidate(g0, g1, mu, ssl[ii], a.rc2)) continue;
            bits |= 1u << ii;
            if (EMIT && n < room) {
                const int c = base + n;
                if (c < a.cap_rec) a.cand[c] = make_int2(j, i0 + ii);
                else atomicOr(a.status, ST_CAPACITY);
            }
            ++n;
        }
        if (!EMIT && a.cand_mask) a.cand_mask[(size_t)(i0 / kSliceChunk) * a.N + j] = bits;
    }
    if (!EMIT && live) a.rec_cnt[j] = n;
    if (EMIT && live)
        for (int k = n; k < room && base + k < a.cap_rec; ++k) a.cand[base + k] = make_int2(j, -1);
}

// Emit pass from the count pass's slab bits (single subject): the block's
// Gaussians own the contiguous candidate range [rec_off[j0], rec_off[j1]); each
// thread places its candidates (slices in order) in shared memory, then the
// block writes the range with consecutive threads on consecutive candidates.
// A range larger than the staging buffer is written directly.
constexpr int kCandThreads = 128;
constexpr int kCandStage = 6144;  // staged candidates per block (48 KB)
__global__ void __launch_bounds__(kCandThreads) k_cand_emit_masks(BinArgs a) {
    extern __shared__ int2 stage[];
    const int j0 = blockIdx.x * kCandThreads, j1 = min(a.N, j0 + kCandThreads);
    const int j = j0 + threadIdx.x;
    const bool live = j < j1;
    const int c0 = a.rec_off[j0], c1 = a.rec_off[j1];
    const bool staged = c1 - c0 <= kCandStage;
    const int base = live ? a.rec_off[j] : 0, room = live ? a.rec_off[j + 1] - base : 0;
    if (live) {
        const int W = (a.M + 31) >> 5;
        int n = 0;
        for (int w = 0; w < W; ++w) {
            unsigned m = a.cand_mask[(size_t)w * a.N + j];
            while (m) {
                const int i = 32 * w + __ffs(m) - 1;
                m &= m - 1u;
                if (n < room) {
                    if (staged) stage[base - c0 + n] = make_int2(j, i);
                    else if (base + n < a.cap_rec) a.cand[base + n] = make_int2(j, i);
                }
                ++n;
            }
        }
        for (int k = n; k < room; ++k) {  // (a count that moved: padding, as the slab pass pads)
            if (staged) stage[base - c0 + k] = make_int2(j, -1);
            else if (base + k < a.cap_rec) a.cand[base + k] = make_int2(j, -1);
        }
    }
    if (!staged) {
        if (live && base + room > a.cap_rec && room > 0) atomicOr(a.status, ST_CAPACITY);
        return;
    }
    __syncthreads();
    for (int c = c0 + threadIdx.x; c < c1; c += kCandThreads) {
        if (c < a.cap_rec) a.cand[c] = stage[c - c0];
        else atomicOr(a.status, ST_CAPACITY);
    }
}

// Thread per candidate: the exact cut, the slice-plane conditioning, the tile
// box and the live-tile count.  Candidates stay the records (same index, so
// the list remains Gaussian-major); candidates that fail hold an empty record
// with no keys.
__global__ void __launch_bounds__(128) k_records(BinArgs a) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_cand = min(*a.n_rec, a.cap_rec);
    if (c >= n_cand) return;
    const int2 ji = a.cand[c];
    const int j = ji.x, i = ji.y;
    bool ok = i >= 0;
    Rec R;
    R.a = make_float4(0.f, 0.f, -1.f, 0.f);
    R.b = make_float4(-1.f, 0.f, -INFINITY, __int_as_float(max(i, 0)));
    int tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0, nk = 0;
    unsigned mask = 0u;
    if (ok) {
        const SliceDev &S = a.slices[i];
        const float mu[3] = {a.theta[j], a.theta[a.N + j], a.theta[2 * a.N + j]};
        const float4 g0 = a.gpre[2 * j], g1 = a.gpre[2 * j + 1];
        RecGeom G;
        ok = rec_geom<true>(g0, g1, mu, S, a.rc2, a.norm_mode, G) &&
             rec_bbox(G, S, a.rc2, a.tile_w, a.tile_h, tx0, tx1, ty0, ty1);
        if (ok) {
            const float L = kNegHalfLog2e;
            R.a = make_float4(G.cb, G.ca, L * G.P2xx * S.dx * S.dx, 2.f * L * G.P2xy * S.dx * S.dy);
            R.b = make_float4(L * G.P2yy * S.dy * S.dy, g1.w * G.w0, L * G.qz, __int_as_float(i));
            nk = count_live_tiles(R, S, tx0, tx1, ty0, ty1, a.tile_w, a.tile_h, a.tile_px_start, a.tile_px_end,
                                  a.qcut, mask);
        }
    }
    a.rec[c] = R;
    a.rec_tiles[c] = make_int2(tx0 | (tx1 << 16), ty0 | (ty1 << 16));
    a.rec_nkeys[c] = nk;
    a.rec_mask[c] = mask;
}

// Keys of one record: exactly the count its record pass found, in row-major
// tile order; should the tile test here come out differently, missing keys are
// padded with the sentinel tile id n_tiles (sorted past every real tile and
// never evaluated) and surplus ones dropped, so the key offsets always hold.
__global__ void k_key_emit(KeyArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_rec = min(*a.n_rec, a.cap_rec);
    if (r >= n_rec) return;
    const int k0 = a.key_off[r];
    const int k1 = k0 + a.rec_nkeys[r];
    if (k1 <= k0) return;
    const int i = a.cand[r].y;  // the record's slice (the full record only when its tiles are tested again)
    const SliceDev &S = a.slices[i];
    const int2 tb = a.rec_tiles[r];
    const int tx0 = tb.x & 0xffff, tx1 = tb.x >> 16, ty0 = tb.y & 0xffff, ty1 = tb.y >> 16;
    unsigned mask = a.rec_mask[r];
    int k = k0;
    if (mask) {  // the record pass's tile tests, row-major bits of the box
        const int wx = tx1 - tx0 + 1;
        while (mask && k < k1) {
            const int b = __ffs(mask) - 1;
            mask &= mask - 1u;
            const int ty = ty0 + b / wx, tx = tx0 + (b - (b / wx) * wx);
            if (k < a.cap_keys) {
                a.keys[k] = (uint32_t)(S.tile_base + ty * S.tiles_x + tx);
                a.key_rec[k] = r;
            } else {
                atomicOr(a.status, ST_CAPACITY);
            }
            ++k;
        }
    } else {
        const Rec R = a.rec[r];
        const float2 iAB = rec_inv_ab(R);
        for (int ty = ty0; ty <= ty1 && k < k1; ++ty)
            for (int tx = tx0; tx <= tx1 && k < k1; ++tx) {
                if (!tile_live(R, iAB, S, tx, ty, a.tile_w, a.tile_h, a.tile_px_start, a.tile_px_end, a.qcut))
                    continue;
                if (k < a.cap_keys) {
                    a.keys[k] = (uint32_t)(S.tile_base + ty * S.tiles_x + tx);
                    a.key_rec[k] = r;
                } else {
                    atomicOr(a.status, ST_CAPACITY);
                }
                ++k;
            }
    }
    for (; k < k1 && k < a.cap_keys; ++k) {  // padding: sentinel tile, zero moments
        a.keys[k] = (uint32_t)a.n_tiles;
        a.key_rec[k] = r;
        if (a.mom) {
            a.mom[2 * k] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.mom[2 * k + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Thread per tile: its run [start, end) in the sorted keys, by two binary
// searches (sentinel keys, tile id n_tiles, sort past every real tile).
__global__ void k_tile_rec_ranges(const uint32_t *__restrict__ keys, const int *n_keys, int cap, int n_tiles,
                                  int *start, int *end) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int n = min(*n_keys, cap);
    auto lower = [&](uint32_t v) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(keys + mid) < v) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    start[t] = lower((uint32_t)t);
    end[t] = lower((uint32_t)t + 1u);
}

// ------------------------------------------------------------- work items
// The sorted (tile, record) list is cut into work items of at most kItemRecs
// records of one tile (a tile with pixels and no records gets one empty item),
// so the evaluation grids are balanced however unevenly records fall on tiles.
// Also counts the forward's tile pairs (sampled pixels x records of each
// tile) into *pairs and *pairs_total when given: one atomic per warp.
__global__ void k_item_count(const int *__restrict__ tps, const int *__restrict__ tpe,
                             const int *__restrict__ trs, const int *__restrict__ tre, int n_tiles,
                             int *__restrict__ cnt, unsigned long long *pairs, unsigned long long *pairs_total) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long np = 0ull;
    if (t < n_tiles) {
        const int npx = tpe[t] - tps[t], nrec = tre[t] - trs[t];
        cnt[t] = npx > 0 ? max(1, (nrec + kItemRecs - 1) / kItemRecs) : 0;
        np = (unsigned long long)max(npx, 0) * (unsigned long long)max(nrec, 0);
    }
    if (!pairs) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) np += __shfl_down_sync(0xffffffffu, np, o);
    if ((threadIdx.x & 31) == 0 && np) {
        atomicAdd(pairs, np);
        if (pairs_total) atomicAdd(pairs_total, np);
    }
}

__global__ void k_item_fill(const int *__restrict__ first, int n_tiles, int *__restrict__ item_tile, int cap) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int e = min(first[t + 1], cap);
    for (int i = first[t]; i < e; ++i) item_tile[i] = t;
}

// Work-queue order key of an item: kItemRecs - its record count, so that a
// stable ascending sort hands out the longest items first (longest processing
// time first bounds the persistent kernels' tail by the shortest items).
__global__ void k_item_key(const int *__restrict__ item_tile, const int *__restrict__ item_first,
                           const int *__restrict__ trs, const int *__restrict__ tre, const int *__restrict__ n_items,
                           int cap, uint32_t *__restrict__ key) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(*n_items, cap)) return;
    const int t = item_tile[i];
    const int rs = trs[t] + (i - item_first[t]) * kItemRecs;
    const int nrec = max(0, min(kItemRecs, tre[t] - rs));
    key[i] = (uint32_t)(kItemRecs - nrec);
}

// ----------------------------------------------------------------- forward
// Tile pixels are addressed densely, (row, col) inside the tile; pixels that are
// not in the sample are evaluated but never read back.
struct TileGeom {
    int x0, y0, rows, cols;
};
__device__ __forceinline__ TileGeom tile_geom(const SliceDev &S, int t, int tw, int th) {
    const int l = t - S.tile_base;
    const int ty = l / S.tiles_x, tx = l - ty * S.tiles_x;
    TileGeom g;
    g.x0 = tx * tw;
    g.y0 = ty * th;
    g.cols = min(tw, S.W - g.x0);
    g.rows = min(th, S.H - g.y0);
    return g;
}

// 16-byte asynchronous global -> shared copies (the forward's record gathers).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Row bands of the forward: 16 consecutive threads of a group (a half-warp)
// own 16 / segs consecutive tile rows.  Bands of a record: those that meet the
// rows of its in-cut box (the rows whose pixel centres can satisfy the cut
// q + log2 w_n >= log2 cutoff_rel, the same box and margin as the backward's);
// its pairs in the other bands are below the cut.  Returns the band bits, 0
// when the box misses the tile's rows.
constexpr int kFwdBands = 16, kFwdBandsMin = 4;
// Floats of the forward's shared per-pixel sums (groups x tile pixels): the
// groups of a 128-thread CTA hold at most 128 x PXR pixels, and a single group
// at most a whole tile (kMaxTilePx).
__host__ __device__ constexpr int fwd_red_floats(int pxr) { return 128 * pxr > kMaxTilePx ? 128 * pxr : kMaxTilePx; }
__host__ __device__ __forceinline__ bool fwd_bands_fit(int tpg, int segs, int threads) {
    return tpg >= 32 && tpg % 16 == 0 && segs <= 16 && 16 % segs == 0 && tpg / 16 <= kFwdBands && threads >= tpg;
}
__device__ __forceinline__ unsigned fwd_band_mask(const Rec &R, float qcut, float by, int rows, int rb) {
    const float kap = R.b.z - qcut;
    const float fa = -R.a.z, fb = -R.b.x, fc = -R.a.w;
    const float D = 4.f * fa * fb - fc * fc;
    if (!(kap >= 0.f && D > 0.f)) return 0u;
    const float ty = fmaxf(4.f * kap * __fdividef(1.f, D) * fa, 0.f);
    const float hy = ty * rsqrtf(fmaxf(ty, 1e-30f)) * 1.001f + 1e-2f;
    const int r0 = max(0, __float2int_ru(fminf(fmaxf(by - hy, -1.f), 64.f)));
    const int r1 = min(rows - 1, __float2int_rd(fminf(fmaxf(by + hy, -1.f), 64.f)));
    if (r0 > r1) return 0u;
    return ((2u << (r1 / rb)) - 1u) & ~((1u << (r0 / rb)) - 1u);
}

// Work item w (queue position) -> item, tile, first record and record count.
struct ItemRef {
    int i, t, rs, nrec;
};
__device__ __forceinline__ ItemRef item_ref(const EvalArgs &a, int w) {
    ItemRef r;
    r.i = a.item_order ? (int)a.item_order[w] : w;
    r.t = a.item_tile[r.i];
    r.rs = a.tile_rec_start[r.t] + (r.i - a.item_first[r.t]) * kItemRecs;
    r.nrec = max(0, min(kItemRecs, a.tile_rec_end[r.t] - r.rs));
    return r;
}

// Persistent CTAs take work items from a queue (Counters::work_fwd) and run a
// software pipeline over them: while item n is evaluated, the records of item
// n + 1 are in flight into shared memory (cp.async, 16 bytes at a time, through
// the item's (record, emit index) references) and the reference list of item
// n + 2 is in flight by one bulk copy (cp.async.bulk, mbarrier completion,
// bounded wait).  The CTA is G groups of threads; in a group each thread owns
// a run of PXR consecutive pixels of one tile row, and the groups split the
// records (every lane of a warp reads the same record: a broadcast).  With the
// row fixed, the record's row terms C2 da and B da^2 are formed once per PXR
// pixels:
//   q = (A db + C2 da) db + B da^2,   sum += w exp2(q).
// Runs of two or more pixels are evaluated two pixels per packed f32x2
// instruction (each lane the IEEE scalar operation).
// The groups' sums meet in shared memory; part[item][pixel] holds the item's
// sum per dense tile pixel and k_fwd_reduce adds a tile's items in item order
// (bitwise reproducible).  COUNT: count sampled pairs inside the cut instead.
// BANDS (tall tiles): each half-warp of a group owns a band of rows and walks
// only the item's records whose in-cut box reaches those rows, from a list per
// band built for every item by a stable ballot compaction (record order, so
// a pixel's sum keeps its order and the output stays bitwise reproducible);
// the lanes of a half-warp still read one record at a time (a broadcast).
template <bool COUNT, int PXR, bool BANDS = false>
__global__ void __launch_bounds__(256) k_fwd_items(EvalArgs a) {
    __shared__ __align__(128) Rec buf[2][kItemRecs];
    __shared__ __align__(16) int2 sref[3][kItemRecs + 2];
    __shared__ __align__(8) uint64_t bar[3];
    __shared__ __align__(8) uint64_t bar_never;  // initialised, never arrived on (test hook only)
    __shared__ __align__(16) float red[fwd_red_floats(PXR)];  // groups x tile pixels
    __shared__ unsigned char present[kMaxTilePx];
    constexpr int NBS = BANDS ? kFwdBands : 1, NRS = BANDS ? kItemRecs : 1;
    __shared__ unsigned char blist[NBS][NRS];  // per row band: its records, in record order
    __shared__ unsigned short bmask[NRS];
    __shared__ int bcnt[BANDS ? kItemRecs / 32 : 1][NBS];
    __shared__ int blen[NBS];
    __shared__ int s_w[3], s_off[3], s_nrec[3], s_pend[3];
    __shared__ int s_fail;
    const int n_items = min(*a.n_items, a.cap_items);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) {
            mbar_init(&bar[k], 1);
            s_pend[k] = 0;
        }
        mbar_init(&bar_never, 1);
        fence_mbar_init();
        s_fail = 0;
    }
    uint32_t phase = 0;  // bit k: parity of bar[k]'s next completion
    unsigned long long useful = 0;
    const int segs = (a.tile_w + PXR - 1) / PXR;
    const int tpg = a.tile_h * segs;
    const int G = max(1, (int)blockDim.x / tpg);
    if (G * a.tile_px > fwd_red_floats(PXR)) {  // (the launcher never picks such a shape; all threads leave)
        if (tid == 0) atomicOr(a.status, ST_SHAPE);
        return;
    }
    const int g = tid / tpg, seg = tid - g * tpg;
    const int row = seg / segs, col0 = (seg - row * segs) * PXR;
    // row bands (packed path): half-warps of 16 / segs rows, when a group is
    // at least a warp and splits into whole half-warp bands
    // (the launcher picks BANDS only for such shapes; NB = 1 otherwise)
    const int NB = (BANDS && !COUNT && PXR >= 2 && fwd_bands_fit(tpg, segs, blockDim.x)) ? tpg / 16 : 1;
    const int RB = NB > 1 ? 16 / segs : a.tile_h;
    // thread 0: take the next queue position into ring slot `slot` and start
    // the bulk copy of its references
    auto take = [&](int slot) {
        const int w = atomicAdd(&a.counters->work_fwd, 1);
        s_w[slot] = w;
        s_nrec[slot] = 0;
        s_off[slot] = 0;
        if (w >= n_items) return;
        const ItemRef ir = item_ref(a, w);
        s_nrec[slot] = ir.nrec;
        if (ir.nrec <= 0) return;
        const int a0 = ir.rs & ~1, off = ir.rs - a0;
        const int cnt = (ir.nrec + off + 1) & ~1;
        s_off[slot] = off;
        s_pend[slot] = 1;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[slot], (uint32_t)cnt * (uint32_t)sizeof(int2));
        bulk_g2s(&sref[slot][0], a.tref + a0, (uint32_t)cnt * (uint32_t)sizeof(int2), &bar[slot]);
    };
    // all threads: wait for slot's references, then start its record copies into buf[b].
    // Under the test hook every block's first such wait is on bar_never instead
    // and runs out after a.wait_test_ns; the copies it skipped are drained below.
    bool test_wait = a.wait_test_ns > 0;
    auto gather = [&](int slot, int b) -> bool {
        const int nrec = s_nrec[slot];
        if (nrec > 0) {
            const bool ok = test_wait ? mbar_wait_bounded(&bar_never, 0u, (uint64_t)a.wait_test_ns)
                                      : mbar_wait_bounded(&bar[slot], (phase >> slot) & 1u, kWaitLimitNs);
            test_wait = false;
            if (!ok) {
                atomicOr(a.status, ST_TIMEOUT);
                s_fail = 1;
                return false;
            }
            phase ^= 1u << slot;
            if (tid == 0) s_pend[slot] = 0;
            const int off = s_off[slot];
            for (int k = tid; k < 2 * nrec; k += blockDim.x) {
                const int r = k >> 1, h = k & 1;
                const Rec *src = a.rec + sref[slot][off + r].x;
                cp_async16(reinterpret_cast<float4 *>(&buf[b][r]) + h, reinterpret_cast<const float4 *>(src) + h);
            }
        }
        cp_async_commit();
        return true;
    };
    __syncthreads();
    if (tid == 0) {
        take(0);
        take(1);
    }
    __syncthreads();
    gather(0, 0);
    for (int n = 0;; ++n) {
        __syncthreads();  // item n - 1 is done: its record buffer and red are free
        const int cur = n % 3, nxt = (n + 1) % 3;
        if (s_fail || s_w[cur] >= n_items) break;
        if (tid == 0) take((n + 2) % 3);
        gather(nxt, (n + 1) & 1);  // item n + 1 (nothing when the queue is empty)
        cp_async_wait<1>();        // item n's records have landed (this thread's copies)
        __syncthreads();           // ... and every thread's
        if (s_fail) break;
        const ItemRef ir = item_ref(a, s_w[cur]);
        const Rec *rb = buf[n & 1];
        const int nrec = ir.nrec;
        const SliceDev &S = a.slices[a.tile_slice[ir.t]];
        const TileGeom tg = tile_geom(S, ir.t, a.tile_w, a.tile_h);
        const bool active = g < G && row < tg.rows;
        const float rowf = (float)(tg.y0 + row) - S.cy0;
        const float colf0 = (float)(tg.x0 + col0) - S.cx0;
        if (BANDS && NB > 1) {
            // per band, the item's records that reach it (stable compaction by
            // ballots over 32-record chunks, so the lists keep record order)
            const int lane = tid & 31;
            const unsigned lt = (1u << lane) - 1u;
            const int nr32 = (nrec + 31) & ~31;
            const float by0 = S.cy0 - (float)tg.y0;  // + the record centre: its tile-local row
            for (int r = tid; r < nr32; r += blockDim.x) {
                const unsigned m = r < nrec ? fwd_band_mask(rb[r], a.qcut, rb[r].a.y + by0, tg.rows, RB) : 0u;
                bmask[r] = (unsigned short)m;
                for (int b = 0; b < NB; ++b) {
                    const unsigned bal = __ballot_sync(0xffffffffu, (m >> b) & 1u);
                    if (lane == 0) bcnt[r >> 5][b] = __popc(bal);
                }
            }
            __syncthreads();
            for (int r = tid; r < nr32; r += blockDim.x) {
                const unsigned m = bmask[r];
                for (int b = 0; b < NB; ++b) {
                    const unsigned bal = __ballot_sync(0xffffffffu, (m >> b) & 1u);
                    if ((m >> b) & 1u) {
                        int off = 0;
                        for (int c = 0; c < (r >> 5); ++c) off += bcnt[c][b];
                        blist[b][off + __popc(bal & lt)] = (unsigned char)r;
                    }
                }
            }
            if (tid < NB) {
                int n = 0;
                for (int c = 0; c < (nr32 >> 5); ++c) n += bcnt[c][tid];
                blen[tid] = n;
            }
            __syncthreads();
        }
        if (COUNT) {
            const int ps = a.tile_px_start[ir.t], pe = a.tile_px_end[ir.t];
            for (int k = tid; k < a.tile_px; k += blockDim.x) present[k] = 0;
            __syncthreads();
            for (int s2 = ps + tid; s2 < pe; s2 += blockDim.x) {
                const int loc = a.sampled[s2] - S.pix_base;
                const int r0 = loc / S.W;
                present[(r0 - tg.y0) * a.tile_w + (loc - r0 * S.W - tg.x0)] = 1;
            }
            __syncthreads();
        }
        float acc[PXR];
#pragma unroll
        for (int k = 0; k < PXR; ++k) acc[k] = 0.f;
        if (active) {
            if (!COUNT && PXR >= 2) {
                // two pixels per packed f32x2 instruction (the scalar loop below is issue
                // bound at 5 slots per pair; packed, the FP32 pipe and MUFU bound it)
                constexpr int H2 = PXR >= 2 ? PXR / 2 : 1;
                float2 colk[H2], acc2[H2];
#pragma unroll
                for (int k = 0; k < H2; ++k) {
                    colk[k] = make_float2(colf0 + (float)(2 * k), colf0 + (float)(2 * k + 1));
                    acc2[k] = make_float2(0.f, 0.f);
                }
                const int band = BANDS && NB > 1 ? seg >> 4 : 0;
                const int len = BANDS && NB > 1 ? blen[band] : nrec;
                for (int i = g; i < len; i += G) {
                    const int r = BANDS && NB > 1 ? (int)blist[band][i] : i;
                    const float4 r0 = rb[r].a;
                    const float4 r1 = rb[r].b;
                    const float dy = rowf - r0.y;
                    const float2 cdy = make_float2(r0.w * dy, r0.w * dy);
                    const float bdy1 = r1.x * dy * dy;
                    const float2 bdy = make_float2(bdy1, bdy1);
                    const float2 az = make_float2(r0.z, r0.z), ncb = make_float2(-r0.x, -r0.x);
                    const float2 w2 = make_float2(r1.y, r1.y);
#pragma unroll
                    for (int k = 0; k < H2; ++k) {
                        const float2 dx = f2_add(colk[k], ncb);
                        const float2 q = f2_fma(f2_fma(az, dx, cdy), dx, bdy);
                        acc2[k] = f2_fma(w2, make_float2(ex2_approx(q.x), ex2_approx(q.y)), acc2[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < H2; ++k) {
                    acc[2 * k] = acc2[k].x;
                    if (2 * k + 1 < PXR) acc[2 * k + 1] = acc2[k].y;
                }
            } else
            for (int r = g; r < nrec; r += G) {
                const float4 r0 = rb[r].a;
                const float4 r1 = rb[r].b;
                const float dy = rowf - r0.y;
                const float cdy = r0.w * dy;
                const float bdy = r1.x * dy * dy;
#pragma unroll
                for (int k = 0; k < PXR; ++k) {
                    const float dx = (colf0 + (float)k) - r0.x;
                    const float q = fmaf(fmaf(r0.z, dx, cdy), dx, bdy);
                    if (!COUNT) {
                        acc[k] = fmaf(r1.y, ex2_approx(q), acc[k]);
                    } else {
                        const int col = col0 + k;
                        useful += (col < tg.cols && present[row * a.tile_w + col] && q + r1.z >= a.qcut) ? 1ull
                                                                                                       : 0ull;
                    }
                }
            }
        }
        if (COUNT) continue;
        // groups -> one sum per dense tile pixel
        if (active) {
            float *dst = red + g * a.tile_px + row * a.tile_w + col0;
            if (PXR % 4 == 0 && ((a.tile_w | a.tile_px) & 3) == 0 && col0 + PXR <= a.tile_w) {
#pragma unroll
                for (int k = 0; k < PXR; k += 4)  // 16-byte stores (4-way fewer bank wavefronts)
                    *reinterpret_cast<float4 *>(dst + k) = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < PXR; ++k)
                    if (col0 + k < a.tile_w) dst[k] = acc[k];
            }
        }
        __syncthreads();
        for (int px = tid; px < a.tile_px; px += blockDim.x) {
            float sum = 0.f;
            for (int gg = 0; gg < G; ++gg) sum += red[gg * a.tile_px + px];
            a.part[(size_t)ir.i * a.tile_px + px] = sum;
        }
    }
    // leave no copy in flight: this thread's record copies, then (thread 0)
    // the outstanding reference copies, each wait bounded
    cp_async_wait<0>();
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < 3; ++k)
            if (s_pend[k]) mbar_wait_bounded(&bar[k], (phase >> k) & 1u, kWaitLimitNs);
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) useful += __shfl_down_sync(0xffffffffu, useful, o);
        if ((tid & 31) == 0 && useful) atomicAdd(a.useful, useful);
    }
}

// Per-slice outlier terms of a pixel of slice i (Sec. 2.4): prediction
// sigma_i * model, loss w (l(r) / omega_i + log omega_i) with l the data term;
// returns dL/dmodel and the pixel's derivatives in log sigma_i and log omega_i
// (slw null: sigma = omega = 1 without the log term).
struct SlwTerms {
    float pred, dLdm, gsig, gomg, loss;
};
__device__ __forceinline__ SlwTerms slw_terms(const float *slw, int M, int i, int l1, float w, float model, float I) {
    const float sig = slw ? expf(slw[i]) : 1.f, lw = slw ? slw[M + i] : 0.f, iw = slw ? expf(-lw) : 1.f;
    SlwTerms t;
    t.pred = sig * model;
    const float r = t.pred - I;
    const float l = l1 ? w * fabsf(r) : w * r * r;
    const float dl = l1 ? w * (float)((r > 0.f) - (r < 0.f)) : 2.f * w * r;
    t.loss = l * iw + (slw ? w * lw : 0.f);
    t.dLdm = sig * dl * iw;
    t.gsig = dl * iw * t.pred;
    t.gomg = w - l * iw;
    return t;
}

// Per tile: add the items' partial sums in order, then residual, dL/dI_hat and loss.
__global__ void __launch_bounds__(kMaxTilePx) k_fwd_reduce(EvalArgs a) {
    __shared__ double red[kMaxTilePx / 32], red_s[kMaxTilePx / 32], red_o[kMaxTilePx / 32];
    __shared__ int rlo[32], rhi[32];  // sampled column range per tile row
    const int t = blockIdx.x;
    const int ps = a.tile_px_start[t], pe = a.tile_px_end[t];
    if (ps >= pe) {
        if (threadIdx.x == 0) {
            a.tile_loss[t] = 0.0;
            if (a.slw) a.slw_tile[2 * t] = a.slw_tile[2 * t + 1] = 0.0;
        }
        return;
    }
    if (threadIdx.x < 32) {
        rlo[threadIdx.x] = 32;
        rhi[threadIdx.x] = -1;
    }
    __syncthreads();
    const int s = ps + threadIdx.x;
    // per-pixel terms in float32, summed over the warp in float32 (fixed
    // order) and over the block's warps in float64: this GPU's float64 rate is
    // a small fraction of its float32 rate
    float l = 0.f, gs = 0.f, go = 0.f;
    if (s < pe) {
        const SliceDev &S = a.slices[a.tile_slice[t]];
        const TileGeom tg = tile_geom(S, t, a.tile_w, a.tile_h);
        const int p = a.sampled[s];
        const int loc = p - S.pix_base;
        const int r0 = loc / S.W;
        const int px = (r0 - tg.y0) * a.tile_w + (loc - r0 * S.W - tg.x0);
        float acc = 0.f;
        const int i1 = min(a.item_first[t + 1], a.cap_items);
        for (int i = a.item_first[t]; i < i1; ++i) acc += a.part[(size_t)i * a.tile_px + px];
        const int64_t ns = a.n_weight > 0 ? a.n_weight : (a.subj_cnt ? a.subj_cnt[S.subject] : *a.n_sampled);
        const float wp = 1.0f / (float)max(ns, (int64_t)1);
        // data term (MSE or L1, subgradient sign(0) = 0) and the per-slice terms
        const SlwTerms st = slw_terms(a.slw, a.M, a.tile_slice[t], a.l1, wp, acc, a.I_obs[p]);
        a.pred[p] = st.pred;
        a.rbar[p] = st.dLdm;
        if (a.tpos_s) a.tpos_s[s] = ((r0 - tg.y0) << 8) | (loc - r0 * S.W - tg.x0);  // for the backward
        atomicMin(&rlo[r0 - tg.y0], loc - r0 * S.W - tg.x0);
        atomicMax(&rhi[r0 - tg.y0], loc - r0 * S.W - tg.x0);
        l = st.loss;
        gs = st.gsig;
        go = st.gomg;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_down_sync(0xffffffffu, l, o);
        gs += __shfl_down_sync(0xffffffffu, gs, o);
        go += __shfl_down_sync(0xffffffffu, go, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = (double)l;
        red_s[threadIdx.x >> 5] = (double)gs;
        red_o[threadIdx.x >> 5] = (double)go;
    }
    __syncthreads();
    if (a.row_rng && threadIdx.x < a.tile_h)
        a.row_rng[t * a.tile_h + threadIdx.x] = make_short2((short)rlo[threadIdx.x], (short)rhi[threadIdx.x]);
    if (threadIdx.x == 0) {
        double sum = 0.0, ss = 0.0, so = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sum += red[w];
            ss += red_s[w];
            so += red_o[w];
        }
        a.tile_loss[t] = sum;
        if (a.slw) {  // per tile; k_slw_slices adds a slice's tiles in tile order
            a.slw_tile[2 * t] = ss;
            a.slw_tile[2 * t + 1] = so;
        }
    }
}

// ---------------------------------------------------------------- backward
// One CTA of kBwdThreads threads per work item (up to kItemRecs = 2 x
// kBwdThreads records of one tile).  A record is evaluated only over its
// in-cut box inside the tile: the rows and columns whose pixel centres can
// satisfy the cut q + log2 w_n >= log2 cutoff_rel (the ellipse's axis-aligned
// half-extents sqrt(4 kappa b / (4ab - c^2)), sqrt(4 kappa a / (4ab - c^2)) of
// the form -q = a db^2 + c db da + b da^2 <= kappa, widened by a margin),
// clipped to the rows and columns of the tile that hold sampled pixels.  Pairs
// outside the box are below the cut, the pairs the method drops.  Rows go two
// at a time through packed f32x2 instructions (lane x row r, lane y row r + 1;
// a row past the box is a tile row, an exact extra term, or past the tile,
// where r_bar reads 0), so a box is ceil(nr / 2) row pairs x nc columns.
// The CTA orders its records by box shape (a counting sort in shared memory:
// row pairs, then columns, largest first); thread t evaluates sorted records t
// and nrec - 1 - t, so the lanes of a warp run loops of the same row-pair and
// column counts and every thread gets one large and one small box.  Which
// thread evaluates a record does not change its moments, so the output does
// not depend on that order.  The tile's r_bar
// (k_rbar_tiles; 0 off the sample) sits in shared memory as pairs of
// vertically adjacent values, one 64-bit load per packed step, with a row
// stride of tile_w + 1 pairs (lanes on different rows spread over the banks).  Per row pair the row terms C da and B da^2 are formed once and
// three packed row sums sum g, g db, g db^2 accumulate (g = r_bar exp2(q));
// they fold into six packed moment sums (sum g, g db, g da, g db^2, g db da,
// g da^2) whose two lanes are added at the end and written to the record's key
// slot.
constexpr int kBwdThreads = kItemRecs / 2;
// Box shape classes: (row pairs 1 .. 16) x (columns 1 .. 32), then the empty box.
constexpr int kBwdClassesMax = 16 * 33 + 1;
// Sorted position class of a packed box, for a tile of nrp_max row pairs.
__device__ __forceinline__ int bwd_class(int box, int nrp_max) {
    if (box == 0) return nrp_max * 33;
    const int nrp = (((box >> 8) & 255) + 1) >> 1, ncol = (box >> 24) & 255;
    return (nrp_max - nrp) * 33 + (32 - ncol);
}

struct __align__(16) BwdRec {  // a record as its evaluating thread reads it
    float cb, ca, A, C;
    float B;
    int box;  // first row | rows << 8 | first column << 16 | columns << 24
    int key;  // emit index of the (tile, record) key: the moment slot
    int pad_;
};

__device__ __forceinline__ int warp_incl_scan_i(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// In-cut box of record R inside the tile (tile-local rows and columns, clipped
// to the sampled range packed in sb), packed as BwdRec::box; 0 when empty.
// The approximate reciprocal and square root are within a few float32 ulps;
// the margin (0.1 % + 0.01 px) covers them.
__device__ __forceinline__ int bwd_box(const Rec &R, float qcut, float bx, float by, int sb) {
    const int rmin = sb & 255, rmax = (sb >> 8) & 255, cmin = (sb >> 16) & 255, cmax = (sb >> 24) & 255;
    const float kap = R.b.z - qcut;  // -q <= kappa inside the cut
    const float fa = -R.a.z, fb = -R.b.x, fc = -R.a.w;
    const float D = 4.f * fa * fb - fc * fc;
    if (!(kap >= 0.f && D > 0.f)) return 0;
    const float s = 4.f * kap * __fdividef(1.f, D);
    const float tx = fmaxf(s * fb, 0.f), ty = fmaxf(s * fa, 0.f);
    const float hx = tx * rsqrtf(fmaxf(tx, 1e-30f)) * 1.001f + 1e-2f;
    const float hy = ty * rsqrtf(fmaxf(ty, 1e-30f)) * 1.001f + 1e-2f;
    const int c0 = max(cmin, __float2int_ru(fminf(fmaxf(bx - hx, -1.f), 64.f)));
    const int c1 = min(cmax, __float2int_rd(fminf(fmaxf(bx + hx, -1.f), 64.f)));
    const int r0 = max(rmin, __float2int_ru(fminf(fmaxf(by - hy, -1.f), 64.f)));
    const int r1 = min(rmax, __float2int_rd(fminf(fmaxf(by + hy, -1.f), 64.f)));
    if (c0 > c1 || r0 > r1) return 0;
    return r0 | ((r1 - r0 + 1) << 8) | (c0 << 16) | ((c1 - c0 + 1) << 24);
}

// Moments of one record over its box (see above); returns the pairs evaluated.
// rb2[row * ts + col] = (r_bar[row][col], r_bar[row + 1][col]).
__device__ __forceinline__ int bwd_eval_rec(const BwdRec &b, const float2 *rb2, int ts, float x0c, float y0c,
                                            float4 *mom) {
    const int r0 = b.box & 255, nr = (b.box >> 8) & 255, c0 = (b.box >> 16) & 255, ncol = (b.box >> 24) & 255;
    float2 m0 = make_float2(0.f, 0.f), m1 = m0, m2 = m0, m3 = m0, m4 = m0, m5 = m0;
    const float2 A2 = make_float2(b.A, b.A), C2 = make_float2(b.C, b.C), B2 = make_float2(b.B, b.B);
    const float2 one = make_float2(1.f, 1.f);
    const float colc = (x0c + (float)c0) - b.cb;
    const float rowc = (y0c + (float)r0) - b.ca;
    const float2 *rp = rb2 + r0 * ts + c0;
    for (int ri = 0; ri < nr; ri += 2, rp += 2 * ts) {
        const float2 dy = make_float2(rowc + (float)ri, rowc + (float)(ri + 1));
        const float2 cc = f2_mul(C2, dy), bb = f2_mul(f2_mul(B2, dy), dy);
        float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, dx = make_float2(colc, colc);
#pragma unroll 2
        for (int j = 0; j < ncol; ++j) {
            const float2 g = rp[j];
            const float2 q = f2_fma(f2_fma(A2, dx, cc), dx, bb);
            const float2 e = f2_mul(g, make_float2(ex2_approx(q.x), ex2_approx(q.y)));
            const float2 ex = f2_mul(e, dx);
            s0 = f2_add(s0, e);
            s1 = f2_add(s1, ex);
            s2 = f2_fma(ex, dx, s2);
            dx = f2_add(dx, one);
        }
        m0 = f2_add(m0, s0);
        m1 = f2_add(m1, s1);
        m3 = f2_add(m3, s2);
        m2 = f2_fma(s0, dy, m2);
        m4 = f2_fma(s1, dy, m4);
        m5 = f2_fma(f2_mul(s0, dy), dy, m5);
    }
    mom[2 * b.key] = make_float4(m0.x + m0.y, m1.x + m1.y, m2.x + m2.y, m3.x + m3.y);
    mom[2 * b.key + 1] = make_float4(m4.x + m4.y, m5.x + m5.y, 0.f, 0.f);
    return ((nr + 1) & ~1) * ncol;
}

__global__ void __launch_bounds__(kBwdThreads, 8) k_bwd_items(EvalArgs a) {
    extern __shared__ float2 rb2[];  // tile_h x (tile_w + 1) pairs (r_bar[row][col], r_bar[row + 1][col])
    __shared__ BwdRec srec[kItemRecs];
    __shared__ int s_item, s_box;
    __shared__ int cls[kBwdClassesMax];  // per class: count, then first sorted position
    __shared__ unsigned long long s_eval;
    const int tid = threadIdx.x;
    const int n_items = min(*a.n_items, a.cap_items);
    const int tw = a.tile_w, th = a.tile_h, ts = tw + 1;
    const int nrp_max = (th + 1) >> 1, ncls = nrp_max * 33 + 1;
    unsigned long long evaluated = 0;
    if (tid == 0) s_eval = 0ull;
    for (;;) {
        __syncthreads();  // previous item's shared buffers are free
        if (tid == 0) s_item = atomicAdd(&a.counters->work_bwd, 1);
        for (int c = tid; c < ncls; c += kBwdThreads) cls[c] = 0;
        __syncthreads();
        if (s_item >= n_items) break;
        const int i = a.item_order ? (int)a.item_order[s_item] : s_item;
        const int t = a.item_tile[i];
        const int ps = a.tile_px_start[t], pe = a.tile_px_end[t];
        const int rs = a.tile_rec_start[t] + (i - a.item_first[t]) * kItemRecs;
        const int nrec = min(kItemRecs, a.tile_rec_end[t] - rs);
        if (ps >= pe || nrec <= 0) continue;
        const SliceDev &S = a.slices[a.tile_slice[t]];
        const TileGeom tg = tile_geom(S, t, tw, th);
        // this thread's records rs + tid and rs + tid + kBwdThreads: loads
        // issued before the r_bar tile is staged
        const bool v0 = tid < nrec, v1 = tid + kBwdThreads < nrec;
        int2 ref0 = make_int2(0, 0), ref1 = ref0;
        Rec R0, R1;
        if (v0) {
            ref0 = a.tref[rs + tid];
            R0 = a.rec[ref0.x];
        }
        if (v1) {
            ref1 = a.tref[rs + tid + kBwdThreads];
            R1 = a.rec[ref1.x];
        }
        const float *rt = a.rbar_tile + (size_t)t * a.tile_px;
        for (int row = tid >> 5; row < th; row += kBwdThreads / 32)  // a warp per row, lanes over columns
            for (int col = tid & 31; col < tw; col += 32)
                rb2[row * ts + col] =
                    make_float2(__ldg(rt + row * tw + col), row + 1 < th ? __ldg(rt + (row + 1) * tw + col) : 0.f);
        if (tid < 32) {  // the tile's rows and columns that hold samples (k_fwd_reduce)
            const short2 rr = tid < th ? a.row_rng[t * th + tid] : make_short2(32, -1);
            const bool has = rr.x <= rr.y;
            const unsigned m = __ballot_sync(0xffffffffu, has);
            const int lo = __reduce_min_sync(0xffffffffu, has ? (int)rr.x : 255);
            const int hi = __reduce_max_sync(0xffffffffu, has ? (int)rr.y : 0);
            if (tid == 0) s_box = (__ffs(m) - 1) | ((31 - __clz(m)) << 8) | (lo << 16) | (hi << 24);
        }
        __syncthreads();
        const float x0c = (float)tg.x0 - S.cx0, y0c = (float)tg.y0 - S.cy0;  // tile origin, slice-centred
        const int sb = s_box;
        int box0 = 0, box1 = 0, cl0 = 0, cl1 = 0, rank0 = 0, rank1 = 0;
        if (v0) {
            box0 = bwd_box(R0, a.qcut, R0.a.x - x0c, R0.a.y - y0c, sb);
            cl0 = bwd_class(box0, nrp_max);
            rank0 = atomicAdd(&cls[cl0], 1);
        }
        if (v1) {
            box1 = bwd_box(R1, a.qcut, R1.a.x - x0c, R1.a.y - y0c, sb);
            cl1 = bwd_class(box1, nrp_max);
            rank1 = atomicAdd(&cls[cl1], 1);
        }
        __syncthreads();
        if (tid < 32) {  // class counts -> first sorted positions (exclusive scan, class order)
            const int per = (ncls + 31) >> 5;
            const int c0 = min(ncls, tid * per), c1 = min(ncls, c0 + per);
            int sum = 0;
            for (int c = c0; c < c1; ++c) sum += cls[c];
            int run = warp_incl_scan_i(sum) - sum;
            for (int c = c0; c < c1; ++c) {
                const int n = cls[c];
                cls[c] = run;
                run += n;
            }
        }
        __syncthreads();
        if (v0) {
            BwdRec b;
            b.cb = R0.a.x;
            b.ca = R0.a.y;
            b.A = R0.a.z;
            b.C = R0.a.w;
            b.B = R0.b.x;
            b.box = box0;
            b.key = ref0.y;
            b.pad_ = 0;
            srec[cls[cl0] + rank0] = b;
        }
        if (v1) {
            BwdRec b;
            b.cb = R1.a.x;
            b.ca = R1.a.y;
            b.A = R1.a.z;
            b.C = R1.a.w;
            b.B = R1.b.x;
            b.box = box1;
            b.key = ref1.y;
            b.pad_ = 0;
            srec[cls[cl1] + rank1] = b;
        }
        __syncthreads();
        // one large and one small box per thread (sorted positions t and nrec - 1 - t)
        if (tid < nrec) evaluated += bwd_eval_rec(srec[tid], rb2, ts, x0c, y0c, a.mom);
        const int u = nrec - 1 - tid;
        if (u >= kBwdThreads) evaluated += bwd_eval_rec(srec[u], rb2, ts, x0c, y0c, a.mom);
    }
    if (a.bwd_pairs_total) {  // pairs this CTA evaluated: one atomic per CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) evaluated += __shfl_down_sync(0xffffffffu, evaluated, o);
        if ((tid & 31) == 0 && evaluated) atomicAdd(&s_eval, evaluated);
        __syncthreads();
        if (tid == 0 && s_eval) atomicAdd(a.bwd_pairs_total, s_eval);
    }
}

// Dense per-tile r_bar for the backward: thread per sample, from the per-pixel
// buffer (a caller may have replaced the forward's values there); the buffer
// is zeroed first, so pixels off the sample hold 0.
__global__ void k_rbar_tiles(EvalArgs a, int cap) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= min(*a.n_sampled, cap)) return;
    const int p = a.sampled[s];
    const int rc = a.tpos_s[s];
    a.rbar_tile[(size_t)a.pix_tile[p] * a.tile_px + (rc >> 8) * a.tile_w + (rc & 255)] = a.rbar[p];
}

// Per-subject losses: block k sums its subject's tiles in tile order.
__global__ void __launch_bounds__(1024) k_loss_reduce(const double *tile_loss, int n, const int *tile_first,
                                                      double *subj_loss) {
    __shared__ double red[32];
    const int k = blockIdx.x;
    const int t0 = tile_first ? tile_first[k] : 0, t1 = tile_first ? tile_first[k + 1] : n;
    double s = 0.0;
    for (int t = t0 + threadIdx.x; t < t1; t += 1024) s += tile_loss[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 32; ++w) tot += red[w];
        subj_loss[k] = tot;
    }
}

__global__ void k_loss_total(const double *subj_loss, int n_subj, double *loss, unsigned *status) {
    double tot = 0.0;
    for (int k = 0; k < n_subj; ++k) tot += subj_loss[k];
    *loss = tot;
    if (!isfinite(tot)) atomicOr(status, ST_NONFINITE);
}

// Sampled pixels per subject (sum of its tiles' pixel counts).
__global__ void __launch_bounds__(256) k_subject_counts(const int *__restrict__ tps, const int *__restrict__ tpe,
                                                       const int *__restrict__ tile_first, int *cnt) {
    __shared__ int red[8];
    const int k = blockIdx.x;
    int s = 0;
    for (int t = tile_first[k] + threadIdx.x; t < tile_first[k + 1]; t += 256) s += tpe[t] - tps[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        cnt[k] = tot;
    }
}

// ------------------------------------------------------------- gradients
// dL/d(record) -> dL/d(m, K) -> Gaussian (mu, Sigma_j, c, log det) and slice
// frame (R_i, t_i).  Moments arrive in slice-centred pixel units about the
// record centre.  A half-warp owns one Gaussian and each of its lanes one of
// the Gaussian's records (records are stored Gaussian-major), so the lanes of
// a half-warp touch distinct slices when they add their slice-frame terms into
// the block's shared-memory accumulators; the 11 Gaussian partials are then
// reduced with half-warp shuffles.
template <typename SLT>
__device__ __forceinline__ void record_chain(const GradArgs &a, int r, const float4 g0, const float4 g1,
                                             const float mu[3], const float Sg[9], float gmu[3], float GS[6],
                                             float &gc, float &glog, float *pacc, int w0, const SLT *slices) {
    float S0 = 0.f, Sx = 0.f, Sy = 0.f, Sxx = 0.f, Sxy = 0.f, Syy = 0.f;
    const int k_end = min(a.key_off[r + 1], a.cap_keys);
    for (int k = max(a.key_off[r], 0); k < k_end; ++k) {
        const float4 u = a.mom[2 * k], v = a.mom[2 * k + 1];
        S0 += u.x;
        Sx += u.y;
        Sy += u.z;
        Sxx += u.w;
        Sxy += v.x;
        Syy += v.y;
    }
    if (S0 == 0.f && Sx == 0.f && Sy == 0.f && Sxx == 0.f && Sxy == 0.f && Syy == 0.f) return;
    const int i = a.cand[r].y;  // the record's slice
    const SLT &SL = slices[i - w0];
    RecGeom G;
    if (!rec_geom<false>(g0, g1, mu, SL, a.rc2, a.norm_mode, G)) return;
    const float dx = SL.dx, dy = SL.dy;
    Sx *= dx;
    Sy *= dy;
    Sxx *= dx * dx;
    Sxy *= dx * dy;
    Syy *= dy * dy;
    const float w = g1.w * G.w0;
    const float Gw = S0 * w;  // dL/d log w
    gc += S0 * G.w0;
    // centre: dL/dc = w P2 S1
    const float Gcx = w * (G.P2xx * Sx + G.P2xy * Sy);
    const float Gcy = w * (G.P2xy * Sx + G.P2yy * Sy);
    // conic: dL/dP2 = -1/2 w S2 -> dL/dM2 = 1/2 w P2 S2 P2
    const float T00 = G.P2xx * Sxx + G.P2xy * Sxy, T01 = G.P2xx * Sxy + G.P2xy * Syy;
    const float T10 = G.P2xy * Sxx + G.P2yy * Sxy, T11 = G.P2xy * Sxy + G.P2yy * Syy;
    const float GMxx = 0.5f * w * (T00 * G.P2xx + T01 * G.P2xy);
    const float GMxy = 0.5f * w * (T00 * G.P2xy + T01 * G.P2yy);
    const float GMyy = 0.5f * w * (T10 * G.P2xy + T11 * G.P2yy);
    const float ik = 1.0f / G.Kzz, kx = G.Kxz, ky = G.Kyz;
    const float mz = G.mz;
    // M2 = K_xy - k k^T / K_zz
    const float Mk0 = GMxx * kx + GMxy * ky, Mk1 = GMxy * kx + GMyy * ky;
    float Gkx = -2.f * Mk0 * ik, Gky = -2.f * Mk1 * ik;
    float Gkap = (kx * Mk0 + ky * Mk1) * ik * ik;
    // centre c = m_xy - k m_z / K_zz
    const float kGc = kx * Gcx + ky * Gcy;
    float Gmz = -kGc * ik;
    Gkx -= Gcx * mz * ik;
    Gky -= Gcy * mz * ik;
    Gkap += kGc * mz * ik * ik;
    // normal weight exp(-1/2 m_z^2 / K_zz)
    Gmz -= Gw * mz * ik;
    Gkap += 0.5f * Gw * mz * mz * ik * ik;
    float GK[9] = {GMxx, GMxy, 0.5f * Gkx, GMxy, GMyy, 0.5f * Gky, 0.5f * Gkx, 0.5f * Gky, Gkap};
    if (a.norm_mode == GSVR_NORM_EXACT) {
        // -1/2 log det K -> -1/2 Gw K^-1 ; 1/2 log det Sigma_j = sum ls -> d ls_k += Gw
        const float c00 = G.Kyy * G.Kzz - G.Kyz * G.Kyz, c01 = G.Kxz * G.Kyz - G.Kxy * G.Kzz;
        const float c02 = G.Kxy * G.Kyz - G.Kxz * G.Kyy, c11 = G.Kxx * G.Kzz - G.Kxz * G.Kxz;
        const float c12 = G.Kxy * G.Kxz - G.Kxx * G.Kyz, c22 = G.Kxx * G.Kyy - G.Kxy * G.Kxy;
        const float idK = 1.0f / (G.Kxx * c00 + G.Kxy * c01 + G.Kxz * c02);
        const float h = -0.5f * Gw * idK;
        GK[0] += h * c00;
        GK[1] += h * c01;
        GK[2] += h * c02;
        GK[3] += h * c01;
        GK[4] += h * c11;
        GK[5] += h * c12;
        GK[6] += h * c02;
        GK[7] += h * c12;
        GK[8] += h * c22;
        glog += Gw;
    }
    const float Gm[3] = {Gcx, Gcy, Gmz};
    const float *R = G.R;
    float RGm[3];
    for (int p = 0; p < 3; ++p) RGm[p] = R[3 * p] * Gm[0] + R[3 * p + 1] * Gm[1] + R[3 * p + 2] * Gm[2];
    for (int p = 0; p < 3; ++p) gmu[p] += RGm[p];
    float RG[9];  // R GK
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            RG[3 * p + q] = R[3 * p] * GK[q] + R[3 * p + 1] * GK[3 + q] + R[3 * p + 2] * GK[6 + q];
    // Sigma_j: R GK R^T (symmetric; xx yy zz xy xz yz)
    auto RGR = [&](int p, int q) { return RG[3 * p] * R[3 * q] + RG[3 * p + 1] * R[3 * q + 1] + RG[3 * p + 2] * R[3 * q + 2]; };
    GS[0] += RGR(0, 0);
    GS[1] += RGR(1, 1);
    GS[2] += RGR(2, 2);
    GS[3] += RGR(0, 1);
    GS[4] += RGR(0, 2);
    GS[5] += RGR(1, 2);
    // slice frame: t -> -R Gm ; R -> d Gm^T + 2 Sigma_j R GK
    float GR[12];
    for (int p = 0; p < 3; ++p) {
        for (int q = 0; q < 3; ++q) {
            const float sm = Sg[3 * p] * RG[q] + Sg[3 * p + 1] * RG[3 + q] + Sg[3 * p + 2] * RG[6 + q];
            GR[3 * p + q] = G.d[p] * Gm[q] + 2.f * sm;
        }
        GR[9 + p] = -RGm[p];
    }
    if (pacc) {
        for (int e = 0; e < 12; ++e) atomicAdd(&pacc[12 * (i - w0) + e], GR[e]);
    } else {
        for (int e = 0; e < 12; ++e) atomicAdd(&a.pose_acc[12 * i + e], (double)GR[e]);
    }
}

// Gaussian epilogue: the summed record gradients v = (d mu (3), d Sigma (xx yy
// zz xy xz yz), d c, d (1/2 log det Sigma)) of Gaussian j -> (mu, ls, q, c)
// through Sigma_j = R(q / |q|) diag(exp(2 ls)) R^T (written to grad).
__device__ __forceinline__ void gauss_epilogue(const GradArgs &a, int j, const float v[11]) {
    const int N = a.N;
    // Sigma_j = Rj diag(s^2) Rj^T -> ls, q (through q / |q|)
    const float GSm[9] = {v[3], v[6], v[7], v[6], v[4], v[8], v[7], v[8], v[5]};
    const float qw = a.theta[6 * N + j], qx = a.theta[7 * N + j], qy = a.theta[8 * N + j], qz = a.theta[9 * N + j];
    const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    const float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
    float Rj[9];
    quat_rot(w, x, y, z, Rj);
    const float s2[3] = {expf(2.f * a.theta[3 * N + j]), expf(2.f * a.theta[4 * N + j]),
                         expf(2.f * a.theta[5 * N + j])};
    float GRj[9];  // GS Rj
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            GRj[3 * p + q] = GSm[3 * p] * Rj[q] + GSm[3 * p + 1] * Rj[3 + q] + GSm[3 * p + 2] * Rj[6 + q];
    float dls[3];
    for (int k = 0; k < 3; ++k) {
        const float d = Rj[k] * GRj[k] + Rj[3 + k] * GRj[3 + k] + Rj[6 + k] * GRj[6 + k];
        dls[k] = 2.f * s2[k] * d + v[10];
    }
    float GRD[9];  // dL/dRj = 2 GS Rj D
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) GRD[3 * p + q] = 2.f * GRj[3 * p + q] * s2[q];
    const float dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const float dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const float dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const float dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    float gq[4] = {0.f, 0.f, 0.f, 0.f};
    for (int e = 0; e < 9; ++e) {
        gq[0] += GRD[e] * dRw[e];
        gq[1] += GRD[e] * dRx[e];
        gq[2] += GRD[e] * dRy[e];
        gq[3] += GRD[e] * dRz[e];
    }
    const float dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    float *g = a.grad;
    g[j] = v[0];
    g[N + j] = v[1];
    g[2 * N + j] = v[2];
    g[3 * N + j] = dls[0];
    g[4 * N + j] = dls[1];
    g[5 * N + j] = dls[2];
    g[6 * N + j] = (gq[0] - w * dot) / qn;
    g[7 * N + j] = (gq[1] - x * dot) / qn;
    g[8 * N + j] = (gq[2] - y * dot) / qn;
    g[9 * N + j] = (gq[3] - z * dot) / qn;
    g[10 * N + j] = v[9];
}

// Warp-centric.  Each block takes a contiguous run of Gaussians (so of at
// most a few subjects) and splits its records evenly over its 8 warps, each
// warp's range starting at a Gaussian's first record (records are stored
// Gaussian-major), so every Gaussian belongs to one warp.  A warp walks its
// range 32 records at a time, a record per lane; the lanes' 11 partial
// Gaussian gradients are summed per Gaussian by a segmented inclusive scan
// over the lanes (shuffles, fixed order: deterministic), a Gaussian that
// continues past the batch carries its partial sum into the next, and the
// lane holding a Gaussian's last record runs the epilogue.  Gaussians without
// records keep the zero the launcher wrote.  Slice-frame gradients go to a
// shared window over the run's subjects' slices, flushed once with float64
// atomics; a block whose window does not fit uses float64 global atomics.
__global__ void __launch_bounds__(256, 3) k_gauss_grad(GradArgs a) {
    extern __shared__ float pacc_s[];  // window x 12
    const int N = a.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (N + gridDim.x - 1) / gridDim.x;
    const int j0 = blockIdx.x * chunk, j1 = min(N, j0 + chunk);
    if (j0 >= j1) return;
    int w0 = 0, w1 = a.M;
    if (a.gauss_subject) {
        w0 = a.subj_slice_first[a.gauss_subject[j0]];
        w1 = a.subj_slice_first[a.gauss_subject[j1 - 1] + 1];
    }
    float *pacc = (w1 - w0) <= a.smem_slices ? pacc_s : nullptr;
    if (pacc) {
        for (int e = tid; e < (w1 - w0) * 12; e += blockDim.x) pacc[e] = 0.f;
    }
    // the window's slice geometry in shared memory when it was given room
    SliceGeo *geo = pacc && a.smem_geo ? reinterpret_cast<SliceGeo *>(pacc_s + 12 * a.smem_slices) : nullptr;
    if (geo) {
        const float *src = reinterpret_cast<const float *>(a.slices + w0);
        float *dst = reinterpret_cast<float *>(geo);
        constexpr int SW = (int)(sizeof(SliceDev) / 4);
        for (int e = tid; e < (w1 - w0) * kSliceGeoWords; e += blockDim.x) {
            const int sl = e / kSliceGeoWords, f = e - sl * kSliceGeoWords;
            dst[e] = src[sl * SW + slice_geo_src(f)];
        }
    }
    __syncthreads();
    auto ro = [&](int j) { return min(a.rec_off[j], a.cap_rec); };
    const int R0 = ro(j0), R1 = ro(j1);
    // first record >= x that starts its Gaussian (R1 if none): whole warp
    auto first_head = [&](int x) {
        for (int base = x; base < R1; base += 32) {
            const int r = base + lane;
            const unsigned hb = __ballot_sync(0xffffffffu, r < R1 && r == ro(a.cand[r].x));
            if (hb) return base + __ffs(hb) - 1;
        }
        return R1;
    };
    const int L = (R1 - R0 + 7) / 8;
    const int rs = warp == 0 ? R0 : first_head(min(R1, R0 + warp * L));
    const int re = warp == 7 ? R1 : first_head(min(R1, R0 + (warp + 1) * L));
    float carry[11];
    int carry_j = -1;
    for (int base = rs; base < re; base += 32) {
        const int r = base + lane;
        const bool valid = r < re;
        const int j = valid ? a.cand[r].x : -2 - lane;  // invalid lanes: segments of their own
        float v[11] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            const float mu[3] = {a.theta[j], a.theta[N + j], a.theta[2 * N + j]};
            const float4 g0 = a.gpre[2 * j], g1 = a.gpre[2 * j + 1];
            const float Sg[9] = {g0.x, g0.w, g1.x, g0.w, g0.y, g1.y, g1.x, g1.y, g0.z};
            if (geo) record_chain(a, r, g0, g1, mu, Sg, v, v + 3, v[9], v[10], pacc, w0, geo);
            else record_chain(a, r, g0, g1, mu, Sg, v, v + 3, v[9], v[10], pacc, w0, a.slices + w0);
        }
        // segmented inclusive scan: lanes of one Gaussian are contiguous
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int ju = __shfl_up_sync(0xffffffffu, j, off);
            const bool same = lane >= off && ju == j;
#pragma unroll
            for (int e = 0; e < 11; ++e) {
                const float vu = __shfl_up_sync(0xffffffffu, v[e], off);
                if (same) v[e] += vu;
            }
        }
        if (j == carry_j) {
#pragma unroll
            for (int e = 0; e < 11; ++e) v[e] += carry[e];
        }
        const int jn = __shfl_down_sync(0xffffffffu, j, 1);
        const bool seg_end = valid && (lane == 31 || jn != j);
        if (seg_end && r + 1 == ro(j + 1)) gauss_epilogue(a, j, v);
        // the Gaussian of lane 31 continues into the next batch unless it ended here
        const int jl = __shfl_sync(0xffffffffu, j, 31);
        const bool cont = __shfl_sync(0xffffffffu, valid && r + 1 < ro(j + 1), 31);
#pragma unroll
        for (int e = 0; e < 11; ++e) carry[e] = __shfl_sync(0xffffffffu, v[e], 31);
        carry_j = cont ? jl : -1;
    }
    if (pacc) {
        __syncthreads();
        for (int e = tid; e < (w1 - w0) * 12; e += blockDim.x) {
            const float val = pacc[e];
            if (val != 0.f) atomicAdd(&a.pose_acc[12 * w0 + e], (double)val);
        }
    }
}

// (R_i, t_i) gradients -> (r, tau): dL/dRod = G_R R0^T + G_t c0^T, and
// dRod/dr_k from the exponential-map derivative of Gallego & Yezzi (2015):
// dR/dr_k = ((r_k [r]x + [r x (I - R) e_k]x) / |r|^2) R, with the first-order
// series [e_k]x + (E_k K + K E_k)/2 near r = 0.
__global__ void k_pose_grad(const double *__restrict__ acc, const SliceStatic *__restrict__ ss,
                            const float *__restrict__ pose, float *__restrict__ gpose, int M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double *A = acc + 12 * i;
    const SliceStatic s = ss[i];
    double G[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            G[3 * a + b] = A[3 * a] * s.R0[3 * b] + A[3 * a + 1] * s.R0[3 * b + 1] + A[3 * a + 2] * s.R0[3 * b + 2] +
                           A[9 + a] * s.c0[b];
    const double r[3] = {pose[6 * i], pose[6 * i + 1], pose[6 * i + 2]};
    const double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double Rr[9];
    rodrigues_d(r, Rr);
    const double K[9] = {0.0, -r[2], r[1], r[2], 0.0, -r[0], -r[1], r[0], 0.0};
    for (int k = 0; k < 3; ++k) {
        double D[9];
        const double e[3] = {k == 0 ? 1.0 : 0.0, k == 1 ? 1.0 : 0.0, k == 2 ? 1.0 : 0.0};
        const double E[9] = {0.0, -e[2], e[1], e[2], 0.0, -e[0], -e[1], e[0], 0.0};
        if (th2 < 1e-14) {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double ek = 0.0, ke = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        ek += E[3 * a + c] * K[3 * c + b];
                        ke += K[3 * a + c] * E[3 * c + b];
                    }
                    D[3 * a + b] = E[3 * a + b] + 0.5 * (ek + ke);
                }
        } else {
            double v[3];  // (I - R) e_k
            for (int a = 0; a < 3; ++a) v[a] = e[a] - Rr[3 * a + k];
            const double c[3] = {r[1] * v[2] - r[2] * v[1], r[2] * v[0] - r[0] * v[2], r[0] * v[1] - r[1] * v[0]};
            const double S[9] = {0.0, -c[2], c[1], c[2], 0.0, -c[0], -c[1], c[0], 0.0};
            double Bm[9];
            for (int e2 = 0; e2 < 9; ++e2) Bm[e2] = (r[k] * K[e2] + S[e2]) / th2;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    D[3 * a + b] = Bm[3 * a] * Rr[b] + Bm[3 * a + 1] * Rr[3 + b] + Bm[3 * a + 2] * Rr[6 + b];
        }
        double g = 0.0;
        for (int e2 = 0; e2 < 9; ++e2) g += G[e2] * D[e2];
        gpose[6 * i + k] = (float)g;
        gpose[6 * i + 3 + k] = (float)A[9 + k];
    }
}

// Adam with StepLR: lr x gamma^((t - 1) / step_every); the 1-based step t from
// the argument or from the device iteration counter (graph replay).
// Adam's per-step scalars (1 / bias corrections, StepLR factor) for a step
// read from the device counter (graph replay), in float64 by one thread.
__global__ void k_adam_scalars(float b1, float b2, int step_every, float gamma, const unsigned long long *d_step,
                               float *scal) {
    const long long t = (long long)(*d_step) + 1;
    scal[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    scal[1] = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
    scal[2] = step_every > 0 ? (float)pow((double)gamma, (double)((t - 1) / step_every)) : 1.0f;
}

__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int N, int M, float lr0, float lr1, float lr2, float lr3, float lr4,
                       float lr5, float b1, float b2, float eps, float ibc1_h, float ibc2_h, float scale_h,
                       const float *__restrict__ d_scal, const uint8_t *__restrict__ frozen) {
    const float s_ibc1 = d_scal ? d_scal[0] : ibc1_h;
    const float s_ibc2 = d_scal ? d_scal[1] : ibc2_h;
    const float s_scale = d_scal ? d_scal[2] : scale_h;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = 11LL * N + 6LL * M;
    if (e >= n) return;
    float lr;
    if (e < 3LL * N) lr = lr0;
    else if (e < 6LL * N) lr = lr1;
    else if (e < 10LL * N) lr = lr2;
    else if (e < 11LL * N) lr = lr3;
    else {
        const int64_t o = e - 11LL * N;
        if (frozen && frozen[o / 6]) return;
        lr = (o % 6) < 3 ? lr4 : lr5;
    }
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    th[e] -= (lr * s_scale) * (mi * s_ibc1) / (sqrtf(vi * s_ibc2) + eps);
}

__global__ void k_advance_step(unsigned long long *d_step) { *d_step += 1ull; }

// ------------------------------------ content-adaptive initialisation (Sec. 2.5)
__device__ __forceinline__ int slice_of_pixel(const SliceDev *__restrict__ sl, int M, int64_t p) {
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)sl[mid].pix_base <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__global__ void k_init_weights(const float *__restrict__ I, const uint8_t *__restrict__ mask,
                               const SliceDev *__restrict__ sl, int M, int64_t P, float lam, int64_t *__restrict__ W) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    if (!mask[p]) {
        W[p] = 0;
        return;
    }
    const SliceDev &S = sl[slice_of_pixel(sl, M, p)];
    const int loc = (int)(p - S.pix_base), row = loc / S.W, col = loc - row * S.W;
    const int cm = max(col - 1, 0), cp = min(col + 1, S.W - 1), rm = max(row - 1, 0), rp = min(row + 1, S.H - 1);
    const float *img = I + S.pix_base;
    // central differences, one-sided at the border; no fused multiply-add anywhere
    float gx = __fdiv_rn(__fsub_rn(img[row * S.W + cp], img[row * S.W + cm]), __fmul_rn(S.dx, (float)(cp - cm)));
    float gy = __fdiv_rn(__fsub_rn(img[rp * S.W + col], img[rm * S.W + col]), __fmul_rn(S.dy, (float)(rp - rm)));
    if (!isfinite(gx)) gx = 0.f;
    if (!isfinite(gy)) gy = 0.f;
    const float g = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
    const float w = __fadd_rn(__fmul_rn(__fsub_rn(1.f, lam), g), lam);
    W[p] = (int64_t)floorf(__fmul_rn(w, 1024.f));
}
// int64 inclusive scan: 4096 per block (256 threads x 16), block totals, offsets
__global__ void __launch_bounds__(256) k_scan64_block(const int64_t *__restrict__ in, int64_t P,
                                                       int64_t *__restrict__ out, int64_t *__restrict__ tot) {
    __shared__ int64_t red[256];
    const int64_t base = (int64_t)blockIdx.x * 4096 + (int64_t)threadIdx.x * 16;
    int64_t v[16], s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = base + k < P ? in[base + k] : 0;
        s += v[k];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {  // inclusive Hillis-Steele over the thread sums
        const int64_t add = threadIdx.x >= o ? red[threadIdx.x - o] : 0;
        __syncthreads();
        red[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t run = red[threadIdx.x] - s;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        run += v[k];
        if (base + k < P) out[base + k] = run;
    }
    if (threadIdx.x == 255) tot[blockIdx.x] = red[255];
}
__global__ void k_scan64_tops(int64_t *tot, int nb) {  // exclusive, one thread (nb is small)
    int64_t run = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t t = tot[b];
        tot[b] = run;
        run += t;
    }
}
__global__ void k_scan64_add(int64_t *__restrict__ out, int64_t P, const int64_t *__restrict__ tot) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) out[p] += tot[p / 4096];
}
__global__ void k_init_draw(const int64_t *__restrict__ C, int64_t P, uint64_t seed, int64_t n,
                            const SliceDev *__restrict__ sl, int M, const float *__restrict__ thick,
                            float *__restrict__ mu, int *__restrict__ pix) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const unsigned long long T = (unsigned long long)C[P - 1];
    const unsigned long long t = __umul64hi(splitmix64_at(seed, (unsigned long long)k), T);
    int64_t lo = 0, hi = P - 1;  // first p with C[p] > t
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((unsigned long long)C[mid] > t) hi = mid;
        else lo = mid + 1;
    }
    const int i = slice_of_pixel(sl, M, lo);
    const SliceDev &S = sl[i];
    const int loc = (int)(lo - S.pix_base), row = loc / S.W, col = loc - row * S.W;
    double j[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        j[a] = (double)(splitmix64_at(seed, (1ull << 40) + 3ull * (unsigned long long)k + a) >> 40) * 0x1p-24 - 0.5;
    const double u0 = ((double)col + j[0] - (double)S.cx0) * (double)S.dx;
    const double u1 = ((double)row + j[1] - (double)S.cy0) * (double)S.dy;
    const double u2 = j[2] * (double)thick[i];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        mu[(size_t)a * n + k] =
            (float)((double)S.R[3 * a] * u0 + (double)S.R[3 * a + 1] * u1 + (double)S.R[3 * a + 2] * u2 + (double)S.t[a]);
    if (pix) pix[k] = (int)lo;
}

__global__ void k_adam_slw(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int M, float lr_sig, float lr_omg, float b1, float b2, float eps,
                           float ibc1_h, float ibc2_h, float scale_h, const float *__restrict__ d_scal,
                           const uint8_t *__restrict__ frozen) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * M) return;
    if (e < M && frozen && frozen[e]) return;  // the reference slice fixes the intensity scale
    const float s_ibc1 = d_scal ? d_scal[0] : ibc1_h, s_ibc2 = d_scal ? d_scal[1] : ibc2_h;
    const float s_scale = d_scal ? d_scal[2] : scale_h;
    const float lr = e < M ? lr_sig : lr_omg;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= (lr * s_scale) * (mi * s_ibc1) / (sqrtf(vi * s_ibc2) + eps);
}
__global__ void k_slw_grad(const double *__restrict__ gacc, int n, float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) grad[e] = (float)gacc[e];
}

// ============================================ normalised top-K forward model
// Eq. 2 with every covariance replaced by its observed covariance (Eq. 4) and
// the ratio of Eq. 5 (sigma_i = 1): I_hat = sum_S c_j E_j / (sum_S E_j + delta),
// E_j = exp(-1/2 v^T Sigma_obs^-1 v), S = the K means nearest the pixel's world
// position (Sec. 2.5, Top-K), ties to the smaller index.  The neighbours come
// from an exact shell search of a uniform grid over the means.


// order-preserving float <-> int for atomic min / max
__device__ __forceinline__ int f2o(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float o2f(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7FFFFFFF); }

__global__ void k_topk_box_init(TopkGrid *g) {
    for (int a = 0; a < 3; ++a) {
        g->box[a] = 0x7FFFFFFF;
        g->box[3 + a] = (int)0x80000000;
    }
}
__global__ void __launch_bounds__(256) k_topk_box(const float *__restrict__ th, int N, TopkGrid *g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int o = j < N ? f2o(th[(size_t)a * N + j]) : 0;
        lo[a] = j < N ? o : 0x7FFFFFFF;
        hi[a] = j < N ? o : (int)0x80000000;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&g->box[a], lo[a]);
            atomicMax(&g->box[3 + a], hi[a]);
        }
}
// cell size h = (box volume x per_cell / N)^(1/3), grown by 10 % steps until the
// cell count fits kTopkMaxCells; cell index = floor((x - org) / h) per axis
__global__ void k_topk_grid_params(TopkGrid *g, int N, float per_cell) {
    float lo[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = o2f(g->box[a]);
        ext[a] = fmaxf(o2f(g->box[3 + a]) - lo[a], 1e-3f);
    }
    float h = cbrtf(ext[0] * ext[1] * ext[2] * per_cell / (float)max(N, 1));
    int n[3];
    for (int it = 0; it < 200; ++it) {
        long long tot = 1;
        for (int a = 0; a < 3; ++a) {
            n[a] = (int)floorf(ext[a] / h) + 1;
            tot *= n[a];
        }
        if (tot <= kTopkMaxCells) break;
        h *= 1.1f;
    }
    for (int a = 0; a < 3; ++a) {
        g->org[a] = lo[a];
        g->n[a] = n[a];
    }
    g->h = h;
    g->inv_h = 1.0f / h;
    g->n_cells = n[0] * n[1] * n[2];
}
__device__ __forceinline__ int topk_cell_axis(const TopkGrid &g, int a, float x) {
    const float f = floorf((x - g.org[a]) * g.inv_h);
    return (int)fminf(fmaxf(f, 0.f), (float)(g.n[a] - 1));
}
__global__ void k_topk_cell_keys(const float *__restrict__ th, int N, const TopkGrid *__restrict__ gp,
                                 uint32_t *__restrict__ keys) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const TopkGrid g = *gp;
    const int cx = topk_cell_axis(g, 0, th[j]), cy = topk_cell_axis(g, 1, th[(size_t)N + j]);
    const int cz = topk_cell_axis(g, 2, th[2 * (size_t)N + j]);
    keys[j] = (uint32_t)((cz * g.n[1] + cy) * g.n[0] + cx);
}
__global__ void k_topk_cell_ranges(const uint32_t *__restrict__ keys, int N, int *__restrict__ start,
                                   int *__restrict__ end) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t c = keys[k];
    if (k == 0 || keys[k - 1] != c) start[c] = k;
    if (k == N - 1 || keys[k + 1] != c) end[c] = k + 1;
}

__global__ void k_topk_gather_means(const float *__restrict__ th, const uint32_t *__restrict__ gidx, int N,
                                    float4 *__restrict__ gm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int j = (int)gidx[k];
    gm[k] = make_float4(th[j], th[(size_t)N + j], th[2 * (size_t)N + j], __int_as_float(j));
}

// The sample's slice (binary search over the slices' first pixels), its world
// position and local coordinate.
struct TopkPixel {
    int i;
    double x[3];  // world position in float64: v = x - mu keeps its low bits far from the origin
    float u[2];
};
__device__ __forceinline__ TopkPixel topk_pixel(const TopkArgs &a, int p) {
    int lo = 0, hi = a.M - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.slices[mid].pix_base <= p) lo = mid;
        else hi = mid - 1;
    }
    TopkPixel q;
    q.i = lo;
    const SliceDev &S = a.slices[lo];
    const int loc = p - S.pix_base, row = loc / S.W, col = loc - row * S.W;
    q.u[0] = ((float)col - S.cx0) * S.dx;
    q.u[1] = ((float)row - S.cy0) * S.dy;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        q.x[k] = (double)S.R[3 * k] * q.u[0] + (double)S.R[3 * k + 1] * q.u[1] + (double)S.t[k];
    return q;
}
// Sigma_obs = Sigma_j + R_i Sigma_PSF R_i^T = L L^T (Cholesky, 3 x 3): the
// quadratic form v^T Sigma_obs^-1 v = |L^-1 v|^2 by forward substitution
// (backward stable, unlike an explicit inverse of an anisotropic Sigma_obs),
// and Sigma_obs^-1 v = L^-T (L^-1 v) by back substitution.
struct TopkChol {
    float i00, l10, l20, i11, l21, i22;  // L with its diagonal stored inverted
};
__device__ __forceinline__ TopkChol topk_chol(const float4 g0, const float4 g1, const float sp[6]) {
    const float a = g0.x + sp[0], d = g0.y + sp[1], f = g0.z + sp[2];
    const float b = g0.w + sp[3], c = g1.x + sp[4], e = g1.y + sp[5];
    TopkChol L;
    const float l00 = sqrtf(a);
    L.i00 = 1.0f / l00;
    L.l10 = b * L.i00;
    L.l20 = c * L.i00;
    const float l11 = sqrtf(fmaxf(d - L.l10 * L.l10, 0.f));
    L.i11 = 1.0f / l11;
    L.l21 = (e - L.l20 * L.l10) * L.i11;
    L.i22 = 1.0f / sqrtf(fmaxf(f - L.l20 * L.l20 - L.l21 * L.l21, 0.f));
    return L;
}
__device__ __forceinline__ void topk_fsub(const TopkChol &L, float vx, float vy, float vz, float w[3]) {
    w[0] = vx * L.i00;
    w[1] = (vy - L.l10 * w[0]) * L.i11;
    w[2] = (vz - L.l20 * w[0] - L.l21 * w[1]) * L.i22;
}
__device__ __forceinline__ void topk_bsub(const TopkChol &L, const float w[3], float z[3]) {
    z[2] = w[2] * L.i22;
    z[1] = (w[1] - L.l21 * z[2]) * L.i11;
    z[0] = (w[0] - L.l10 * z[1] - L.l20 * z[2]) * L.i00;
}
// R diag(var) R^T of a slice (symmetric 6)
__device__ __forceinline__ void topk_psf(const SliceDev &S, float sp[6]) {
    auto e = [&](int p, int q) {
        return S.R[3 * p] * S.var[0] * S.R[3 * q] + S.R[3 * p + 1] * S.var[1] * S.R[3 * q + 1] +
               S.R[3 * p + 2] * S.var[2] * S.R[3 * q + 2];
    };
    sp[0] = e(0, 0);
    sp[1] = e(1, 1);
    sp[2] = e(2, 2);
    sp[3] = e(0, 1);
    sp[4] = e(0, 2);
    sp[5] = e(1, 2);
}

// Forward: a warp per sample.  Block b owns samples [128 b, 128 b + 128); its
// warp w takes samples 128 b + w, + 4, ... in order.  The K nearest means of
// the sample's world position x are kept in shared memory as a sorted list of
// 64-bit keys (d^2 bits << 32 | j): ordering keys orders by (d^2, j), the
// smaller index winning ties.  Candidates are the cell-ordered means of the
// last grid build; the lanes test 32 at a time (one 16-byte read each)
// against the list's largest key (every candidate passes
// until the list holds K); the passing keys are sorted across the warp by a
// shuffle bitonic network and merged into the list by ranks (binary searches),
// keeping the K smallest; passing keys are staged and merged 32 at a time, and
// before each stopping test.  Distances are float32 about the corner of x's cell
// (x - o in float64 once per sample, mu - o in float32 per candidate: errors of
// a few 1e-7 mm at millimetre distances).  Cells are visited in shells of
// Chebyshev distance 0, 1, 2, ... around x's cell, 32 cells of a shell at a
// time (lane l tests cell l and reads its range; each round takes one
// candidate of its own cell per lane); once the list is full a cell whose box
// lies farther than its largest distance is skipped unread; the search stops
// when the list is full and its largest distance is at most the distance from
// x to the nearest face of the scanned box with grid cells beyond it (every
// unscanned mean lies beyond such a face), or when no such face is left.  The ratio
// is then formed over the neighbours in parallel across the lanes, with
// float64 sums reduced in a fixed order.
constexpr int kTopkWarps = kTopkThreads / 32;

struct TopkList {
    unsigned long long *cur, *alt;  // sorted keys (cur) and the merge target (alt)
    unsigned long long *stage;      // the round's sorted keys (32)
    int cnt;                        // keys held (warp-uniform)
    unsigned long long tau;         // largest key when cnt == K, else all ones
};

// Merge a set of passing keys (one per lane, all ones where none) into the list.
__device__ __forceinline__ void topk_merge(TopkList &T, unsigned long long v, int m, int K, int lane) {
    // ascending bitonic sort of the 32 lanes' keys (all-ones keys sort last)
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, stride);
            const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
            v = (lower == up) ? (v < o ? v : o) : (v < o ? o : v);
        }
    T.stage[lane] = v;
    __syncwarp();
    const int n = T.cnt;
    // the round's key i goes to i + (list keys below it)
    if (lane < m) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (T.cur[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        const int pos = lane + lo;
        if (pos < K) T.alt[pos] = v;
    }
    // list key e goes to e + (round keys below it)
    for (int e = lane; e < n; e += 32) {
        const unsigned long long x = T.cur[e];
        int lo = 0, hi = m;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (T.stage[mid] < x) lo = mid + 1;
            else hi = mid;
        }
        const int pos = e + lo;
        if (pos < K) T.alt[pos] = x;
    }
    __syncwarp();
    unsigned long long *t = T.cur;
    T.cur = T.alt;
    T.alt = t;
    T.cnt = min(n + m, K);
    T.tau = T.cnt == K ? T.cur[K - 1] : ~0ull;
    __syncwarp();
}

__global__ void __launch_bounds__(kTopkThreads) k_topk_fwd(TopkArgs a) {
    __shared__ unsigned long long s_list[kTopkWarps][2][kTopkMaxK];
    __shared__ unsigned long long s_stage[kTopkWarps][32];
    __shared__ unsigned long long s_pend[kTopkWarps][64];  // passing keys not merged yet
    __shared__ double red[kTopkWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ns = min(*a.n_sampled, a.cap_px);
    const int N = a.N, K = a.K;
    double lsum = 0.0;  // lane 0: this warp's losses, in sample order
    for (int t = w; t < kTopkThreads; t += kTopkWarps) {
        const int s = blockIdx.x * kTopkThreads + t;
        if (s >= ns) break;
        const int p = a.sampled[s];
        const TopkPixel q = topk_pixel(a, p);
        TopkList T{s_list[w][0], s_list[w][1], s_stage[w], 0, ~0ull};
        if (N > 0) {  // (no grid is built without Gaussians)
            const TopkGrid g = *a.grid;
            int c[3];
            float o[3], xo[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                c[k] = topk_cell_axis(g, k, (float)q.x[k]);
                o[k] = g.org[k] + (float)c[k] * g.h;
                xo[k] = (float)(q.x[k] - (double)o[k]);
            }
            // passing keys are staged and merged 32 at a time (and before every
            // stopping test), so the list's largest key tightens at each merge
            unsigned long long *P = s_pend[w];
            int pc = 0;
            auto flush = [&]() {
                for (int h = 0; h < pc; h += 32) {
                    const int m = min(pc - h, 32);
                    topk_merge(T, lane < m ? P[h + lane] : ~0ull, m, K, lane);
                }
                pc = 0;
            };
            for (int sh = 0;; ++sh) {
                // the cells of shell sh (Chebyshev distance sh from c, clipped to
                // the grid), 32 at a time: lane l tests and reads cell l of the batch
                int lo3[3], n3[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    lo3[k] = max(c[k] - sh, 0);
                    n3[k] = min(c[k] + sh, g.n[k] - 1) - lo3[k] + 1;
                }
                const int total = n3[0] * n3[1] * n3[2];
                for (int b0 = 0; b0 < total; b0 += 32) {
                    const int idx = b0 + lane;
                    int k0 = 0, k1 = 0;
                    if (idx < total) {
                        const int cx = lo3[0] + idx % n3[0], cy = lo3[1] + (idx / n3[0]) % n3[1];
                        const int cz = lo3[2] + idx / (n3[0] * n3[1]);
                        const int cc[3] = {cx, cy, cz};
                        const int cheb = max(max(abs(cx - c[0]), abs(cy - c[1])), abs(cz - c[2]));
                        bool take = cheb == sh;
                        if (take && T.cnt == K) {  // prune: squared distance from x to the cell's box
                            float m2 = 0.f;
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const float lo = (float)(cc[k] - c[k]) * g.h, hi = lo + g.h;
                                const float dk = fmaxf(fmaxf(lo - xo[k], xo[k] - hi), 0.f);
                                m2 = fmaf(dk, dk, m2);
                            }
                            take = m2 <= __uint_as_float((unsigned)(T.tau >> 32)) * (1.0f + 1e-5f);
                        }
                        if (take) {
                            const int cell = (cz * g.n[1] + cy) * g.n[0] + cx;
                            k0 = a.cell_start[cell];
                            k1 = a.cell_end[cell];
                        }
                    }
                    // rounds: one candidate of its own cell per lane
                    const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)(k1 - k0));
                    for (int r = 0; r < rounds; ++r) {
                        const int k = k0 + r;
                        unsigned long long key = ~0ull;
                        if (k < k1) {
                            const float4 m = a.gm[k];
                            const float vx = xo[0] - (m.x - o[0]), vy = xo[1] - (m.y - o[1]), vz = xo[2] - (m.z - o[2]);
                            const float d2 = fmaf(vz, vz, fmaf(vy, vy, vx * vx));
                            key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)__float_as_int(m.w);
                        }
                        const bool pass = key < T.tau;
                        const unsigned bal = __ballot_sync(0xffffffffu, pass);
                        if (bal) {
                            if (pass) P[pc + __popc(bal & ((1u << lane) - 1u))] = key;
                            pc += __popc(bal);
                            __syncwarp();
                            if (pc >= 32) flush();
                        }
                    }
                }
                if (pc > 0) flush();
                // unscanned cells lie beyond the faces of the scanned box that have
                // grid cells beyond them; rho = distance from x to the nearest such face
                bool all = true;
                float rho = 3.4e38f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (c[k] - sh > 0) {
                        all = false;
                        rho = fminf(rho, xo[k] + (float)sh * g.h);
                    }
                    if (c[k] + sh < g.n[k] - 1) {
                        all = false;
                        rho = fminf(rho, (float)(sh + 1) * g.h - xo[k]);
                    }
                }
                if (all) break;
                if (T.cnt == K && rho > 0.f && __uint_as_float((unsigned)(T.tau >> 32)) <= rho * rho) break;
            }
        }
        // the ratio over the neighbours, lanes in parallel
        const int cnt = T.cnt;
        const SliceDev &S = a.slices[q.i];
        float sp[6];
        topk_psf(S, sp);
        double num = 0.0, den = 0.0;
        for (int e = lane; e < cnt; e += 32) {
            const int j = (int)(unsigned)(T.cur[e] & 0xffffffffull);
            const float4 g0 = a.gpre[2 * j], g1 = a.gpre[2 * j + 1];
            const TopkChol L = topk_chol(g0, g1, sp);
            float wv[3];
            topk_fsub(L, (float)(q.x[0] - (double)a.theta[j]), (float)(q.x[1] - (double)a.theta[(size_t)N + j]),
                      (float)(q.x[2] - (double)a.theta[2 * (size_t)N + j]), wv);
            const float E = expf(-0.5f * (wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]));
            num += (double)g1.w * (double)E;
            den += (double)E;
            a.nbr[(size_t)s * K + e] = j;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, off);
            den += __shfl_xor_sync(0xffffffffu, den, off);
        }
        if (lane == 0) {
            a.ncnt[s] = cnt;
            const float D = (float)(den + (double)a.delta);
            const float Ih = (float)(num / (den + (double)a.delta));
            const float wp = 1.0f / (float)(a.n_weight > 0 ? a.n_weight : (int64_t)max(ns, 1));
            const SlwTerms st = slw_terms(a.slw, a.M, q.i, a.l1, wp, Ih, a.I_obs[p]);
            a.pred[p] = st.pred;
            a.rbar[p] = st.dLdm;
            a.pstat[s] = make_float2(Ih, D);  // the ratio before sigma_i: the backward's I_hat
            lsum += st.loss;
            if (a.slw) {
                atomicAdd(&a.slw_gacc[q.i], (double)st.gsig);
                atomicAdd(&a.slw_gacc[a.M + q.i], (double)st.gomg);
            }
        }
        __syncwarp();  // the list is free for the next sample
    }
    if (lane == 0) red[w] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < kTopkWarps; ++k) tot += red[k];
        a.loss_part[blockIdx.x] = tot;
    }
}
__global__ void __launch_bounds__(256) k_topk_loss_total(const double *__restrict__ part, int nb, double *loss,
                                                         unsigned *status) {
    __shared__ double red[8];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) s += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        *loss = t;
        if (!isfinite(t)) atomicOr(status, ST_NONFINITE);
    }
}

// Backward: thread per sample.  With gbar = dL/dI_hat, D = sum E + delta and
// gam = gbar (c_j - I_hat) / D * E_j (dL/dE_j times E_j), per neighbour:
//   dL/dc_j += gbar E_j / D,  dL/dmu_j += gam P v,  dL/dSigma_j += 1/2 gam P v v^T P,
//   dL/dx -= gam P v (pixel position), and Sigma_obs's R_i S R_i^T term gives
//   dL/dR_i += 2 G R_i diag(var) with G the summed dL/dSigma_obs; x = R_i u + t_i
//   gives dL/dR_i += dL/dx u^T, dL/dt_i += dL/dx.
// A block's samples are consecutive in tile order, so they share most
// neighbours: per-Gaussian sums go to a shared-memory hash table (open
// addressing, kTopkHash slots) and per-slice sums to a small table, flushed with
// one global atomic per (block, Gaussian, component); an insertion that finds
// no slot adds to global memory directly.
constexpr int kTopkHash = 1024, kTopkPoseSlots = 8;
__global__ void __launch_bounds__(kTopkThreads) k_topk_bwd(TopkArgs a) {
    __shared__ int hk[kTopkHash];
    __shared__ float hv[10][kTopkHash];
    __shared__ int pk[kTopkPoseSlots];
    __shared__ float pv[12][kTopkPoseSlots];
    const int tid = threadIdx.x, N = a.N, K = a.K;
    for (int e = tid; e < kTopkHash; e += kTopkThreads) {
        hk[e] = -1;
#pragma unroll
        for (int c = 0; c < 10; ++c) hv[c][e] = 0.f;
    }
    if (tid < kTopkPoseSlots) {
        pk[tid] = -1;
#pragma unroll
        for (int c = 0; c < 12; ++c) pv[c][tid] = 0.f;
    }
    __syncthreads();
    const int ns = min(*a.n_sampled, a.cap_px);
    const int s = blockIdx.x * kTopkThreads + tid;
    if (s < ns) {
        const int p = a.sampled[s];
        const TopkPixel q = topk_pixel(a, p);
        const SliceDev &S = a.slices[q.i];
        float sp[6];
        topk_psf(S, sp);
        const float2 st = a.pstat[s];
        const float Ih = st.x, D = st.y, gbar = a.rbar[p];
        float gx[3] = {0.f, 0.f, 0.f}, Go[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int cnt = a.ncnt[s];
        for (int e = 0; e < cnt; ++e) {
            const int j = a.nbr[(size_t)s * K + e];
            const float4 g0 = a.gpre[2 * j], g1 = a.gpre[2 * j + 1];
            const TopkChol L = topk_chol(g0, g1, sp);
            float w[3], z[3];
            topk_fsub(L, (float)(q.x[0] - (double)a.theta[j]), (float)(q.x[1] - (double)a.theta[(size_t)N + j]),
                      (float)(q.x[2] - (double)a.theta[2 * (size_t)N + j]), w);
            topk_bsub(L, w, z);
            const float px = z[0], py = z[1], pz = z[2];  // Sigma_obs^-1 v
            const float E = expf(-0.5f * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
            const float gam = gbar * (g1.w - Ih) / D * E;
            const float hg = 0.5f * gam;
            float val[10] = {gam * px, gam * py, gam * pz, hg * px * px, hg * py * py, hg * pz * pz,
                             hg * px * py, hg * px * pz, hg * py * pz, gbar * E / D};
            gx[0] -= val[0];
            gx[1] -= val[1];
            gx[2] -= val[2];
#pragma unroll
            for (int c = 0; c < 6; ++c) Go[c] += val[3 + c];
            // shared slot of Gaussian j
            unsigned hh = ((unsigned)j * 2654435761u) >> (32 - 10);
            int slot = -1;
            for (int probe = 0; probe < 64; ++probe) {
                const int old = atomicCAS(&hk[hh], -1, j);
                if (old == -1 || old == j) {
                    slot = (int)hh;
                    break;
                }
                hh = (hh + 1) & (kTopkHash - 1);
            }
            if (slot >= 0) {
#pragma unroll
                for (int c = 0; c < 10; ++c) atomicAdd(&hv[c][slot], val[c]);
            } else {
#pragma unroll
                for (int c = 0; c < 10; ++c) atomicAdd(&a.gacc[(size_t)c * N + j], val[c]);
            }
        }
        // slice frame: dL/dR_i = dL/dx u^T + 2 G R diag(var), dL/dt_i = dL/dx
        const float Gm[9] = {Go[0], Go[3], Go[4], Go[3], Go[1], Go[5], Go[4], Go[5], Go[2]};
        float GR[12];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const float GRS = Gm[3 * r] * S.R[cc] + Gm[3 * r + 1] * S.R[3 + cc] + Gm[3 * r + 2] * S.R[6 + cc];
                GR[3 * r + cc] = 2.f * GRS * S.var[cc] + gx[r] * (cc < 2 ? q.u[cc] : 0.f);
            }
        GR[9] = gx[0];
        GR[10] = gx[1];
        GR[11] = gx[2];
        int slot = -1;
        for (int probe = 0; probe < kTopkPoseSlots; ++probe) {
            const int hh = (q.i + probe) & (kTopkPoseSlots - 1);
            const int old = atomicCAS(&pk[hh], -1, q.i);
            if (old == -1 || old == q.i) {
                slot = hh;
                break;
            }
        }
        if (slot >= 0) {
#pragma unroll
            for (int c = 0; c < 12; ++c) atomicAdd(&pv[c][slot], GR[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 12; ++c) atomicAdd(&a.pose_acc[12 * q.i + c], (double)GR[c]);
        }
    }
    __syncthreads();
    for (int e = tid; e < kTopkHash; e += kTopkThreads) {
        const int j = hk[e];
        if (j < 0) continue;
#pragma unroll
        for (int c = 0; c < 10; ++c) {
            const float v = hv[c][e];
            if (v != 0.f) atomicAdd(&a.gacc[(size_t)c * N + j], v);
        }
    }
    if (tid < kTopkPoseSlots && pk[tid] >= 0) {
#pragma unroll
        for (int c = 0; c < 12; ++c) atomicAdd(&a.pose_acc[12 * pk[tid] + c], (double)pv[c][tid]);
    }
}
__global__ void k_topk_epilogue(GradArgs a, const float *__restrict__ gacc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.N) return;
    float v[11];
#pragma unroll
    for (int c = 0; c < 10; ++c) v[c] = gacc[(size_t)c * a.N + j];
    v[10] = 0.f;  // no log-determinant factor in the ratio
    gauss_epilogue(a, j, v);
}

__global__ void __launch_bounds__(1024) k_scale_reg_loss(const float *__restrict__ th, int N, float lambda,
                                                          float s_target, double *loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (int e = threadIdx.x; e < 3 * N; e += 1024) {
        const double d = (double)expf(th[(size_t)3 * N + e]) - (double)s_target;
        s += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += red[w];
        *loss += (double)lambda * t;
    }
}
__global__ void k_scale_reg_grad(const float *__restrict__ th, int N, float lambda, float s_target,
                                 float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * N) return;
    const float sc = expf(th[(size_t)3 * N + e]);
    grad[(size_t)3 * N + e] += 2.f * lambda * (sc - s_target) * sc;
}

inline int cdiv(int64_t a, int b) { return (int)((a + b - 1) / b); }

std::atomic<long long> g_launches{0};
inline void counted(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace

long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ launchers
void launch_gauss_prep(const float *theta, int N, float4 *gpre, unsigned *status, cudaStream_t st) {
    if (N <= 0) return;
    k_gauss_prep<<<cdiv(N, 256), 256, 0, st>>>(theta, N, gpre, status);
    counted();
}
void launch_pose_prep(const float *pose, const SliceStatic *ss, SliceDev *sd, int M, unsigned *status,
                      cudaStream_t st) {
    if (M <= 0) return;
    // float64-bound per slice: spread the slices over the SMs (one per block
    // while they are fewer than the SMs)
    const int bs = std::max(1, std::min(128, cdiv(M, 148)));
    k_pose_prep<<<cdiv(M, bs), bs, 0, st>>>(pose, ss, sd, M, status);
    counted();
}
void launch_cand_count(const BinArgs &a, cudaStream_t st) {
    if (a.N <= 0) return;
    k_cand<false><<<cdiv(a.N, 128), 128, 0, st>>>(a);
    counted();
}
void launch_cand_emit(const BinArgs &a, cudaStream_t st) {
    if (a.N <= 0) return;
    if (a.cand_mask && !a.gauss_subject) {
        static int attr_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (attr_dev != dev) {
            cudaFuncSetAttribute(k_cand_emit_masks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kCandStage * sizeof(int2)));
            attr_dev = dev;
        }
        k_cand_emit_masks<<<cdiv(a.N, kCandThreads), kCandThreads, kCandStage * sizeof(int2), st>>>(a);
    } else {
        k_cand<true><<<cdiv(a.N, 128), 128, 0, st>>>(a);
    }
    counted();
}
void launch_records(const BinArgs &a, int n_cand_max, cudaStream_t st) {
    if (n_cand_max <= 0) return;
    k_records<<<cdiv(n_cand_max, 128), 128, 0, st>>>(a);
    counted();
}
void launch_key_emit(const KeyArgs &a, int n_rec_max, cudaStream_t st) {
    if (n_rec_max <= 0) return;
    k_key_emit<<<cdiv(n_rec_max, 256), 256, 0, st>>>(a);
    counted();
}
void launch_tile_rec_ranges(const uint32_t *keys, const int *n_keys, int cap_keys, int n_tiles, int *start, int *end,
                            cudaStream_t st) {
    // every tile is written, also when there are no keys (cap_keys 0: empty ranges, keys never read)
    if (n_tiles <= 0) return;
    k_tile_rec_ranges<<<cdiv(n_tiles, 256), 256, 0, st>>>(keys, n_keys, std::max(cap_keys, 0), n_tiles, start, end);
    counted();
}
static inline int round_warp(int n) { return (n + 31) / 32 * 32; }
void launch_items(const int *tps, const int *tpe, const int *trs, const int *tre, int n_tiles, int *cnt,
                  const int *first, int *item_tile, int cap_items, int phase, cudaStream_t st,
                  unsigned long long *pairs, unsigned long long *pairs_total) {
    if (n_tiles <= 0) return;
    if (phase == 0)
        k_item_count<<<cdiv(n_tiles, 256), 256, 0, st>>>(tps, tpe, trs, tre, n_tiles, cnt, pairs, pairs_total);
    else k_item_fill<<<cdiv(n_tiles, 256), 256, 0, st>>>(first, n_tiles, item_tile, cap_items);
    counted();
}
void launch_item_order(const int *item_tile, const int *item_first, const int *trs, const int *tre,
                       const int *n_items, int cap_items, uint32_t *key, uint32_t *key_sorted, uint32_t *order,
                       const SortScratch &ss, cudaStream_t st) {
    if (cap_items <= 0) return;
    k_item_key<<<cdiv(cap_items, 256), 256, 0, st>>>(item_tile, item_first, trs, tre, n_items, cap_items, key);
    counted();
    int bits = 1;
    while ((1 << bits) <= kItemRecs) ++bits;
    radix_sort_pairs(key, nullptr, key_sorted, order, n_items, cap_items, bits, ss, st);
}
// Forward pixels per thread: the requested run (1, 2, 4, 8 or 16), else the
// whole row for tiles 13 to 16 wide (on the 1M-Gaussian workload at 16 x 16 the
// forward takes 5.23 ms with 16-pixel runs, 5.62 ms with 8), 8 for wider tiles
// (32 x 32: 8.83 ms against 9.36 with 16, as finer row bands cull more), 4 for
// tiles 12 wide and 2 below: the row terms amortised over the longest run.
int fwd_pxr(int tile_w, int req) {
    if (req == 1 || req == 2 || req == 4 || req == 8 || req == 16) return req;
    return tile_w > 16 ? 8 : (tile_w > 12 ? 16 : (tile_w == 12 ? 4 : 2));
}
// Forward CTA shape: groups of tile_h x ceil(tile_w / PXR) threads, as many
// groups as fit in 128 threads (at least one).
int fwd_threads(int tile_w, int tile_h, int pxr) {
    const int tpg = tile_h * ((tile_w + pxr - 1) / pxr);
    const int G = std::max(1, 128 / tpg);
    return round_warp(G * tpg);
}
bool fwd_shape_fits(int tile_w, int tile_h, int pxr) {
    const int tpg = tile_h * ((tile_w + pxr - 1) / pxr);
    const int G = std::max(1, fwd_threads(tile_w, tile_h, pxr) / tpg);
    return G * tile_w * tile_h <= fwd_red_floats(pxr);
}
int eval_blocks_per_sm(int tile_w, int tile_h, bool backward, int pxr_req) {
    int nb = 0;
    if (backward) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bwd_items, kBwdThreads,
                                                      (size_t)tile_h * (tile_w + 1) * sizeof(float2));
    } else {
        const int pxr = fwd_pxr(tile_w, pxr_req);
        const int nt = fwd_threads(tile_w, tile_h, pxr);
        if (pxr == 16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_items<false, 16>, nt, 0);
        else if (pxr == 8) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_items<false, 8>, nt, 0);
        else if (pxr == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_items<false, 4>, nt, 0);
        else if (pxr == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_items<false, 2>, nt, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fwd_items<false, 1>, nt, 0);
    }
    cudaGetLastError();
    return std::max(nb, 1);
}
static int n_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}
// Persistent grid: n_SM x the requested CTAs per SM (at most as many as fit;
// all that fit when not requested), never more CTAs than items.  A request of
// -1 launches one CTA per item slot instead (the hardware schedules the CTAs;
// each takes one item from the queue, the surplus ones find it empty).
static int eval_grid(const EvalArgs &a, bool backward) {
    const int req = backward ? a.bwd_bps : a.fwd_bps;
    if (req < 0) return std::max(1, a.cap_items);
    const int fit = eval_blocks_per_sm(a.tile_w, a.tile_h, backward, a.fwd_pxr);
    const int g = n_sms() * (req > 0 ? std::min(req, fit) : fit);
    return std::max(1, std::min(g, a.cap_items));
}
template <bool COUNT>
static void fwd_items(const EvalArgs &a, cudaStream_t st) {
    const int pxr = fwd_pxr(a.tile_w, a.fwd_pxr);
    const int nt = fwd_threads(a.tile_w, a.tile_h, pxr);
    cudaMemsetAsync(&a.counters->work_fwd, 0, sizeof(int), st);
    const int grid = eval_grid(a, false);
    // row bands from kFwdBandsMin bands up: on the 1M-Gaussian workload the lists
    // cut the forward 13.1 -> 8.8 ms at 32 x 32 (8 bands) and 8.5 -> 7.0-7.4 ms
    // at 32 x 16 / 16 x 32 (4 bands), and cost 7-10 % with 2 bands
    const int segs = (a.tile_w + pxr - 1) / pxr;
    const int tpg = a.tile_h * segs;
    const bool bands = !COUNT && pxr >= 2 && fwd_bands_fit(tpg, segs, nt) && tpg / 16 >= kFwdBandsMin;
    if (pxr == 16 && bands) k_fwd_items<COUNT, 16, true><<<grid, nt, 0, st>>>(a);
    else if (pxr == 16) k_fwd_items<COUNT, 16><<<grid, nt, 0, st>>>(a);
    else if (pxr == 8 && bands) k_fwd_items<COUNT, 8, true><<<grid, nt, 0, st>>>(a);
    else if (pxr == 4 && bands) k_fwd_items<COUNT, 4, true><<<grid, nt, 0, st>>>(a);
    else if (pxr == 2 && bands) k_fwd_items<COUNT, 2, true><<<grid, nt, 0, st>>>(a);
    else if (pxr == 8) k_fwd_items<COUNT, 8><<<grid, nt, 0, st>>>(a);
    else if (pxr == 4) k_fwd_items<COUNT, 4><<<grid, nt, 0, st>>>(a);
    else if (pxr == 2) k_fwd_items<COUNT, 2><<<grid, nt, 0, st>>>(a);
    else k_fwd_items<COUNT, 1><<<grid, nt, 0, st>>>(a);
    counted();
}
void launch_forward(const EvalArgs &a, cudaStream_t st) {
    if (a.n_tiles <= 0) return;
    if (a.cap_items > 0) fwd_items<false>(a, st);
    k_fwd_reduce<<<a.n_tiles, round_warp(a.tile_px), 0, st>>>(a);
    counted();
}
void launch_count_pairs(const EvalArgs &a, cudaStream_t st) {
    if (a.n_tiles <= 0 || a.cap_items <= 0) return;
    fwd_items<true>(a, st);
}
void launch_backward(const EvalArgs &a, int cap_px, cudaStream_t st) {
    if (a.n_tiles <= 0 || a.cap_items <= 0) return;
    cudaMemsetAsync(a.rbar_tile, 0, sizeof(float) * (size_t)a.n_tiles * a.tile_px, st);
    if (cap_px > 0) {
        k_rbar_tiles<<<cdiv(cap_px, 256), 256, 0, st>>>(a, cap_px);
        counted();
    }
    cudaMemsetAsync(&a.counters->work_bwd, 0, sizeof(int), st);
    k_bwd_items<<<eval_grid(a, true), kBwdThreads, (size_t)a.tile_h * (a.tile_w + 1) * sizeof(float2), st>>>(a);
    counted();
}
void launch_loss_reduce(const double *tile_loss, int n_tiles, const int *tile_first, int n_subj, double *subj_loss,
                        double *loss, unsigned *status, cudaStream_t st) {
    k_loss_reduce<<<std::max(n_subj, 1), 1024, 0, st>>>(tile_loss, n_tiles, tile_first, subj_loss);
    k_loss_total<<<1, 1, 0, st>>>(subj_loss, std::max(n_subj, 1), loss, status);
    counted(2);
}
void launch_subject_counts(const int *tps, const int *tpe, const int *tile_first, int n_subj, int *cnt,
                           cudaStream_t st) {
    if (n_subj <= 0) return;
    k_subject_counts<<<n_subj, 256, 0, st>>>(tps, tpe, tile_first, cnt);
    counted();
}
void launch_gauss_grad(const GradArgs &a, cudaStream_t st) {
    if (a.N <= 0) return;
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 148;
    }
    GradArgs g = a;
    const int blocks = std::min(cdiv((int64_t)a.N * 16, 256), n_sm * 3);  // one wave at 3 CTAs / SM
    // the widest slice window of any block (the kernel's chunking, on the host)
    int widest = a.M;
    if (a.gauss_subject && a.h_gauss_first && a.h_slice_first && a.n_subj > 1) {
        const int chunk = (a.N + blocks - 1) / blocks;
        auto subject_of = [&](int64_t j) {
            return (int)(std::upper_bound(a.h_gauss_first, a.h_gauss_first + a.n_subj + 1, j) - a.h_gauss_first) - 1;
        };
        widest = 0;
        for (int b = 0; b < blocks; ++b) {
            const int64_t j0 = (int64_t)b * chunk, j1 = std::min<int64_t>(a.N, j0 + chunk);
            if (j0 >= j1) break;
            widest = std::max(widest, a.h_slice_first[subject_of(j1 - 1) + 1] - a.h_slice_first[subject_of(j0)]);
        }
    }
    g.smem_slices = std::min(widest, a.smem_slices);
    // the slice geometry joins the accumulators when both fit in 96 KB
    g.smem_geo = (size_t)g.smem_slices * (12 + kSliceGeoWords) * sizeof(float) <= 96 * 1024;
    const size_t smem = (size_t)g.smem_slices * (12 + (g.smem_geo ? kSliceGeoWords : 0)) * sizeof(float);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_gauss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // Gaussians without records get no epilogue: their gradient is this zero
    cudaMemsetAsync(g.grad, 0, sizeof(float) * 11 * (size_t)a.N, st);
    k_gauss_grad<<<blocks, 256, smem, st>>>(g);
    counted();
}
void launch_pose_grad(const double *pose_acc, const SliceStatic *ss, const float *pose, float *grad_pose, int M,
                      cudaStream_t st) {
    if (M <= 0) return;
    const int bs = std::max(1, std::min(64, cdiv(M, 148)));
    k_pose_grad<<<cdiv(M, bs), bs, 0, st>>>(pose_acc, ss, pose, grad_pose, M);
    counted();
}
void launch_adam(float *theta, const float *grad, float *m, float *v, int N, int M, const float lr[6], float b1,
                 float b2, float eps, int step_every, float gamma, long long t_host, const unsigned long long *d_step,
                 float *d_scal, const uint8_t *frozen, cudaStream_t st) {
    const int64_t n = 11LL * N + 6LL * M;
    if (n <= 0) return;
    float h[3] = {1.f, 1.f, 1.f};
    if (d_step) {
        k_adam_scalars<<<1, 1, 0, st>>>(b1, b2, step_every, gamma, d_step, d_scal);
        counted();
    } else {
        h[0] = (float)(1.0 / (1.0 - std::pow((double)b1, (double)t_host)));
        h[1] = (float)(1.0 / (1.0 - std::pow((double)b2, (double)t_host)));
        h[2] = step_every > 0 ? (float)std::pow((double)gamma, (double)((t_host - 1) / step_every)) : 1.0f;
    }
    k_adam<<<cdiv(n, 256), 256, 0, st>>>(theta, grad, m, v, N, M, lr[0], lr[1], lr[2], lr[3], lr[4], lr[5], b1, b2,
                                         eps, h[0], h[1], h[2], d_step ? d_scal : nullptr, frozen);
    counted();
}
void launch_adam_slw(float *p, const float *g, float *m, float *v, int M, float lr_sig, float lr_omg, float b1,
                     float b2, float eps, int step_every, float gamma, long long t_host, const unsigned long long *d_step,
                     const float *d_scal, const uint8_t *frozen, cudaStream_t st) {
    if (M <= 0) return;
    float h[3] = {1.f, 1.f, 1.f};
    if (!d_step) {
        h[0] = (float)(1.0 / (1.0 - std::pow((double)b1, (double)t_host)));
        h[1] = (float)(1.0 / (1.0 - std::pow((double)b2, (double)t_host)));
        h[2] = step_every > 0 ? (float)std::pow((double)gamma, (double)((t_host - 1) / step_every)) : 1.0f;
    }
    k_adam_slw<<<cdiv(2LL * M, 256), 256, 0, st>>>(p, g, m, v, M, lr_sig, lr_omg, b1, b2, eps, h[0], h[1], h[2],
                                                   d_step ? d_scal : nullptr, frozen);
    counted();
}
void launch_init_weights(const float *I, const uint8_t *mask, const SliceDev *slices, int M, int64_t P, float lam,
                         int64_t *W, int64_t *C, int64_t *scratch, cudaStream_t st) {
    if (P <= 0) return;
    const int nb = cdiv(P, 4096);
    k_init_weights<<<cdiv(P, 256), 256, 0, st>>>(I, mask, slices, M, P, lam, W);
    k_scan64_block<<<nb, 256, 0, st>>>(W, P, C, scratch);
    k_scan64_tops<<<1, 1, 0, st>>>(scratch, nb);
    k_scan64_add<<<cdiv(P, 256), 256, 0, st>>>(C, P, scratch);
    counted(4);
}
void launch_init_draw(const int64_t *C, int64_t P, uint64_t seed, int64_t n, const SliceDev *slices, int M,
                      const float *thickness, float *mu, int *pix, cudaStream_t st) {
    if (n <= 0 || P <= 0) return;
    k_init_draw<<<cdiv(n, 256), 256, 0, st>>>(C, P, seed, n, slices, M, thickness, mu, pix);
    counted();
}
// Per slice: the gradients of log sigma_i and log omega_i, the sums of its
// tiles' terms in tile order (bitwise reproducible).
__global__ void k_slw_slices(const double *__restrict__ slw_tile, const SliceDev *__restrict__ slices, int M,
                             double *__restrict__ gacc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const SliceDev &S = slices[i];
    double gs = 0.0, go = 0.0;
    for (int t = S.tile_base; t < S.tile_base + S.tiles_x * S.tiles_y; ++t) {
        gs += slw_tile[2 * t];
        go += slw_tile[2 * t + 1];
    }
    gacc[i] = gs;
    gacc[M + i] = go;
}
void launch_slw_slices(const double *slw_tile, const SliceDev *slices, int M, double *gacc, cudaStream_t st) {
    if (M <= 0) return;
    k_slw_slices<<<cdiv(M, 128), 128, 0, st>>>(slw_tile, slices, M, gacc);
    counted();
}
void launch_slw_grad(const double *gacc, int n, float *grad, cudaStream_t st) {
    if (n <= 0) return;
    k_slw_grad<<<cdiv(n, 256), 256, 0, st>>>(gacc, n, grad);
    counted();
}
void launch_advance_step(unsigned long long *d_step, cudaStream_t st) {
    k_advance_step<<<1, 1, 0, st>>>(d_step);
    counted();
}
void launch_sample_flags(int n_subj, const int *mask_first, const int *out_first, int n_out, uint64_t seed,
                         uint64_t step, const unsigned long long *d_step, const int *mask_tpos, int *flags,
                         cudaStream_t st) {
    if (n_out <= 0) return;
    k_sample_flags<<<cdiv(n_out, 256), 256, 0, st>>>(n_subj, mask_first, out_first, n_out, seed, step, d_step,
                                                     mask_tpos, flags);
    counted();
}
void launch_flags_from_list(const int *idx, int n, int n_pix, const uint8_t *mask, const int *pix_tpos,
                            int *flags, unsigned *status, cudaStream_t st) {
    if (n <= 0) return;
    k_flags_from_list<<<cdiv(n, 256), 256, 0, st>>>(idx, n, n_pix, mask, pix_tpos, flags, status);
    counted();
}
void launch_flags_from_list_rank(const int *idx, int n, int n_pix, const int *pix_mrank, int *flags,
                                 unsigned *status, cudaStream_t st) {
    if (n <= 0) return;
    k_flags_from_list_rank<<<cdiv(n, 256), 256, 0, st>>>(idx, n, n_pix, pix_mrank, flags, status);
    counted();
}
void launch_compact(const int *flags, const int *pos, const int *tile_sorted_pix, int n_pix, int *sampled,
                    cudaStream_t st) {
    if (n_pix <= 0) return;
    k_compact<<<cdiv(n_pix, 256), 256, 0, st>>>(flags, pos, tile_sorted_pix, n_pix, sampled);
    counted();
}
void launch_tile_px_ranges(const int *sampled, const int *n_sampled, int cap, const int *pix_tile, int *start,
                           int *end, cudaStream_t st) {
    if (cap <= 0) return;
    k_tile_px_ranges<<<cdiv(cap, 256), 256, 0, st>>>(sampled, n_sampled, cap, pix_tile, start, end);
    counted();
}
void launch_set_count(int *dst, int v, cudaStream_t st) {
    k_set_count<<<1, 1, 0, st>>>(dst, v);
    counted();
}

void launch_topk_grid(const float *theta, int N, float per_cell, TopkGrid *g, uint32_t *keys, cudaStream_t st) {
    if (N <= 0) return;
    k_topk_box_init<<<1, 1, 0, st>>>(g);
    k_topk_box<<<cdiv(N, 256), 256, 0, st>>>(theta, N, g);
    k_topk_grid_params<<<1, 1, 0, st>>>(g, N, per_cell);
    k_topk_cell_keys<<<cdiv(N, 256), 256, 0, st>>>(theta, N, g, keys);
    counted(4);
}
void launch_topk_cell_ranges(const uint32_t *keys_sorted, int N, int *cell_start, int *cell_end, cudaStream_t st) {
    if (N <= 0) return;
    k_topk_cell_ranges<<<cdiv(N, 256), 256, 0, st>>>(keys_sorted, N, cell_start, cell_end);
    counted();
}
void launch_scale_reg_loss(const float *theta, int N, float lambda, float s_target, double *loss, cudaStream_t st) {
    if (N <= 0) return;
    k_scale_reg_loss<<<1, 1024, 0, st>>>(theta, N, lambda, s_target, loss);
    counted();
}
void launch_scale_reg_grad(const float *theta, int N, float lambda, float s_target, float *grad, cudaStream_t st) {
    if (N <= 0) return;
    k_scale_reg_grad<<<cdiv(3LL * N, 256), 256, 0, st>>>(theta, N, lambda, s_target, grad);
    counted();
}
void launch_topk_gather_means(const float *theta, const uint32_t *gidx, int N, float4 *gm, cudaStream_t st) {
    if (N <= 0) return;
    k_topk_gather_means<<<cdiv(N, 256), 256, 0, st>>>(theta, gidx, N, gm);
    counted();
}
void launch_topk_forward(const TopkArgs &a, int cap_px, double *loss, cudaStream_t st) {
    const int nb = std::max(1, cdiv(cap_px, kTopkThreads));
    k_topk_fwd<<<nb, kTopkThreads, 0, st>>>(a);
    k_topk_loss_total<<<1, 256, 0, st>>>(a.loss_part, nb, loss, a.status);
    counted(2);
}
void launch_topk_backward(const TopkArgs &a, int cap_px, cudaStream_t st) {
    const int nb = std::max(1, cdiv(cap_px, kTopkThreads));
    k_topk_bwd<<<nb, kTopkThreads, 0, st>>>(a);
    counted();
}
void launch_topk_epilogue(const float *theta, const float *gacc, int N, float *grad, cudaStream_t st) {
    if (N <= 0) return;
    GradArgs g{};
    g.theta = theta;
    g.N = N;
    g.grad = grad;
    k_topk_epilogue<<<cdiv(N, 256), 256, 0, st>>>(g, gacc);
    counted();
}
void note_launches(int n) { counted(n); }

}  // namespace gsvr
