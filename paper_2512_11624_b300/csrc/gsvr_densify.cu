// gsvr_densify.cu -- coarse-to-fine densification of the Gaussians: split,
// clone and prune (the progressive densification the paper names as future
// work, after the adaptive density control of 3D Gaussian Splatting).
//
// Statistics: per Gaussian the running sums of ||dL/dmu_j|| and dL/dmu_j over
// the backward passes since the last densification (float4 per Gaussian) and
// the pass count.  Decisions are float32 comparisons of the mean norm and of
// the largest log-scale, so they are reproducible bit for bit.  Output order
// is the input order, a split or cloned Gaussian giving two adjacent children
// (an exclusive scan of the per-Gaussian output counts places them).
#include <algorithm>
#include "gsvr_launch.cuh"

namespace gsvr {

namespace {

constexpr int kDensThreads = 256;

__global__ void __launch_bounds__(kDensThreads) k_dens_accum(const float *__restrict__ grad, int N, float4 *__restrict__ acc,
                                                         int *__restrict__ cnt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) cnt[0] += 1;
    if (j >= N) return;
    const float gx = grad[j], gy = grad[N + j], gz = grad[2 * N + j];
    // ((gx gx + gy gy) + gz gz), each operation rounded on its own
    const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz)));
    float4 a = acc[j];
    a.x = __fadd_rn(a.x, n);
    a.y = __fadd_rn(a.y, gx);
    a.z = __fadd_rn(a.z, gy);
    a.w = __fadd_rn(a.w, gz);
    acc[j] = a;
}

__global__ void __launch_bounds__(kDensThreads) k_dens_decide(const float *__restrict__ theta, int N,
                                                          const float4 *__restrict__ acc, const int *__restrict__ cnt,
                                                          float tau_g, float tau_ls, float eps_c,
                                                          uint8_t *__restrict__ kind, int *__restrict__ nout,
                                                          int *__restrict__ counts) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const float c = theta[10 * N + j];
    int k;
    if (fabsf(c) < eps_c) {
        k = kDensPrune;
    } else {
        const int ct = cnt[0];
        const float avg = ct > 0 ? __fdiv_rn(acc[j].x, (float)ct) : 0.f;
        if (avg > tau_g) {
            const float lmax = fmaxf(fmaxf(theta[3 * N + j], theta[4 * N + j]), theta[5 * N + j]);
            k = lmax > tau_ls ? kDensSplit : kDensClone;
        } else {
            k = kDensKeep;
        }
    }
    kind[j] = (uint8_t)k;
    nout[j] = k == kDensPrune ? 0 : (k == kDensKeep ? 1 : 2);
    if (k == kDensSplit) atomicAdd(counts + 0, 1);
    if (k == kDensClone) atomicAdd(counts + 1, 1);
    if (k == kDensPrune) atomicAdd(counts + 2, 1);
}

__global__ void __launch_bounds__(kDensThreads) k_dens_emit(const float *__restrict__ theta, const float *__restrict__ m,
                                                        const float *__restrict__ v, int N, const float4 *__restrict__ acc,
                                                        const uint8_t *__restrict__ kind, const int *__restrict__ off,
                                                        int N2, DensParams p, float *__restrict__ theta2,
                                                        float *__restrict__ m2, float *__restrict__ v2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int k = kind[j];
    if (k == kDensPrune) return;
    const int o = off[j];
    if (k == kDensKeep) {
#pragma unroll
        for (int e = 0; e < 11; ++e) {
            theta2[e * N2 + o] = theta[e * N + j];
            m2[e * N2 + o] = m[e * N + j];
            v2[e * N2 + o] = v[e * N + j];
        }
        return;
    }
    float mu[3], ls[3], q[4];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        mu[e] = theta[e * N + j];
        ls[e] = theta[(3 + e) * N + j];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) q[e] = theta[(6 + e) * N + j];
    const float c = theta[10 * N + j];
    // principal axis: the rotation's column of the largest log-scale (first on ties)
    int ax = 0;
    float best = ls[0];
    if (ls[1] > best) {
        ax = 1;
        best = ls[1];
    }
    if (ls[2] > best) ax = 2;
    const float qi = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] * qi, x = q[1] * qi, y = q[2] * qi, z = q[3] * qi;
    float a[3];
    if (ax == 0) {
        a[0] = 1.f - 2.f * (y * y + z * z);
        a[1] = 2.f * (x * y + w * z);
        a[2] = 2.f * (x * z - w * y);
    } else if (ax == 1) {
        a[0] = 2.f * (x * y - w * z);
        a[1] = 1.f - 2.f * (x * x + z * z);
        a[2] = 2.f * (y * z + w * x);
    } else {
        a[0] = 2.f * (x * z + w * y);
        a[1] = 2.f * (y * z - w * x);
        a[2] = 1.f - 2.f * (x * x + y * y);
    }
    float step[3], c2;
    if (k == kDensSplit) {
        const float d = expf(ls[ax]) * p.split_offset;
#pragma unroll
        for (int e = 0; e < 3; ++e) step[e] = d * a[e];
        ls[ax] -= p.log_split_factor;
        c2 = p.mass_preserving ? c * p.split_factor * 0.5f : c;
    } else {
        const float4 g = acc[j];
        const float n2 = g.y * g.y + g.z * g.z + g.w * g.w;
        float u[3] = {a[0], a[1], a[2]};
        if (n2 > 0.f) {
            const float ni = rsqrtf(n2);
            u[0] = g.y * ni;
            u[1] = g.z * ni;
            u[2] = g.w * ni;
        }
        const float d = p.clone_offset * expf(fminf(fminf(ls[0], ls[1]), ls[2]));
#pragma unroll
        for (int e = 0; e < 3; ++e) step[e] = d * u[e];
        c2 = p.mass_preserving ? 0.5f * c : c;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = o + h;
        const float sg = h == 0 ? 1.f : -1.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            theta2[e * N2 + t] = mu[e] + sg * step[e];
            theta2[(3 + e) * N2 + t] = ls[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) theta2[(6 + e) * N2 + t] = q[e];
        theta2[10 * N2 + t] = c2;
#pragma unroll
        for (int e = 0; e < 11; ++e) {
            m2[e * N2 + t] = 0.f;
            v2[e * N2 + t] = 0.f;
        }
    }
}

}  // namespace

void launch_dens_accum(const float *grad, int N, float4 *acc, int *cnt, cudaStream_t st) {
    k_dens_accum<<<(std::max(N, 1) + kDensThreads - 1) / kDensThreads, kDensThreads, 0, st>>>(grad, N, acc, cnt);
    note_launches(1);
}

void launch_dens_decide(const float *theta, int N, const float4 *acc, const int *cnt, float tau_g, float tau_ls,
                        float eps_c, uint8_t *kind, int *nout, int *counts, cudaStream_t st) {
    if (N <= 0) return;
    k_dens_decide<<<(N + kDensThreads - 1) / kDensThreads, kDensThreads, 0, st>>>(theta, N, acc, cnt, tau_g, tau_ls, eps_c, kind,
                                                                      nout, counts);
    note_launches(1);
}

void launch_dens_emit(const float *theta, const float *m, const float *v, int N, const float4 *acc,
                      const uint8_t *kind, const int *off, int N2, const DensParams &p, float *theta2, float *m2,
                      float *v2, cudaStream_t st) {
    if (N <= 0) return;
    k_dens_emit<<<(N + kDensThreads - 1) / kDensThreads, kDensThreads, 0, st>>>(theta, m, v, N, acc, kind, off, N2, p, theta2, m2,
                                                                    v2);
    note_launches(1);
}

}  // namespace gsvr
