// gsvr_cnn.cu -- the slice-pose regression network (include/gsvr_cnn.h):
// 3x3 / stride-2 convolutions as implicit GEMMs on the bfloat16 tensor cores
// (mma.sync m16n8k16, float32 accumulation, operands staged through shared
// memory and read with ldmatrix), the float32 head, the loss and Adam.
//
// Convolution as GEMM, rows m = (b, oh, ow), columns k = (kh, kw, ci):
//   forward  Y[m][co]   = sum_k X(m, k) W[co][k]             (X = im2col of x)
//   dgrad    D[m][k]    = sum_co G[m][co] W[co][k], then dx gathers D (col2im)
//   wgrad    dW[co][k]  = sum_m G[m][co] X(m, k), the bias as an extra column
// One GEMM kernel serves the three: its operand loaders produce 8 consecutive
// reduction-index values of one row (16 bytes) and its epilogue consumes the
// float32 accumulators.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <vector>

#include "gsvr_cnn.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128, BN = 64, BK = 32, LDS = BK + 8, GT = 256;
constexpr int kImage = GSVR_CNN_IMAGE, kAux = GSVR_CNN_AUX, kOut = GSVR_CNN_OUT, kHidden = 256;
constexpr int kLayers = 6;
constexpr int kCh[kLayers + 1] = {1, 32, 64, 128, 256, 256, 512};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }
__device__ __forceinline__ uint4 pack8(const bf16 v[8]) {
    uint4 u;
    uint32_t *p = reinterpret_cast<uint32_t *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        p[i] = (uint32_t)__bfloat16_as_ushort(v[2 * i]) | ((uint32_t)__bfloat16_as_ushort(v[2 * i + 1]) << 16);
    return u;
}

struct ConvShape {
    int B, H, W, Ci, OH, OW, Co;
};

// ---------------------------------------------------------------- loaders
// Each returns the 8 bfloat16 values (row, k0 .. k0 + 7) of its operand;
// entries with row >= rows or k >= k_end read 0.

// X(m, k) = x[b][2 oh - 1 + kh][2 ow - 1 + kw][ci] (zero padding); Ci % 8 == 0.
struct LoadIm2col {
    const bf16 *x;
    ConvShape s;
    int rows, K;
    __device__ uint4 operator()(int m, int k0, int k_end) const {
        if (m >= rows || k0 >= k_end) return zero4();
        const int tap = k0 / s.Ci, ci = k0 - tap * s.Ci;
        const int kh = tap / 3, kw = tap - 3 * kh;
        const int ow = m % s.OW, t = m / s.OW, oh = t % s.OH, b = t / s.OH;
        const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
        if (ih < 0 || ih >= s.H || iw < 0 || iw >= s.W) return zero4();
        return *reinterpret_cast<const uint4 *>(x + (((size_t)b * s.H + ih) * s.W + iw) * s.Ci + ci);
    }
};

// Row-major matrix p[row][ld] (ld % 8 == 0, 16-byte aligned rows).
struct LoadRows {
    const bf16 *p;
    int rows, ld;
    __device__ uint4 operator()(int r, int k0, int k_end) const {
        if (r >= rows || k0 >= k_end) return zero4();
        return *reinterpret_cast<const uint4 *>(p + (size_t)r * ld + k0);
    }
};

// Transposed access: value (r, k) = p[k][r] of a row-major p[.][ld].
struct LoadCols {
    const bf16 *p;
    int rows, ld;
    __device__ uint4 operator()(int r, int k0, int k_end) const {
        bf16 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v[i] = (r < rows && k0 + i < k_end) ? p[(size_t)(k0 + i) * ld + r] : __float2bfloat16(0.f);
        return pack8(v);
    }
};

// Transposed im2col: value (k, m) = X(m, k) for k < K, 1 for k == K (the bias
// column), 0 beyond.
struct LoadIm2colT {
    const bf16 *x;
    ConvShape s;
    int K;
    __device__ uint4 operator()(int k, int m0, int m_end) const {
        bf16 v[8];
        if (k > K) return zero4();
        if (k == K) {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __float2bfloat16(m0 + i < m_end ? 1.f : 0.f);
            return pack8(v);
        }
        const int tap = k / s.Ci, ci = k - tap * s.Ci;
        const int kh = tap / 3, kw = tap - 3 * kh;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = m0 + i;
            v[i] = __float2bfloat16(0.f);
            if (m < m_end) {
                const int ow = m % s.OW, t = m / s.OW, oh = t % s.OH, b = t / s.OH;
                const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
                if (ih >= 0 && ih < s.H && iw >= 0 && iw < s.W)
                    v[i] = x[(((size_t)b * s.H + ih) * s.W + iw) * s.Ci + ci];
            }
        }
        return pack8(v);
    }
};

// ---------------------------------------------------------------- epilogues
struct EpiConv {  // y = bf16(relu?(acc + bias)), y32 = the float value
    bf16 *y;
    float *y32;
    const float *bias;
    int rows, cols, relu;
    __device__ void operator()(int r, int c, float v) const {
        if (r >= rows || c >= cols) return;
        v += bias ? bias[c] : 0.f;
        if (relu) v = fmaxf(v, 0.f);
        y[(size_t)r * cols + c] = __float2bfloat16(v);
        if (y32) y32[(size_t)r * cols + c] = v;
    }
};
struct EpiStore {  // out[r][ld] = acc
    float *out;
    int rows, cols, ld;
    __device__ void operator()(int r, int c, float v) const {
        if (r < rows && c < cols) out[(size_t)r * ld + c] = v;
    }
};
struct EpiWgrad {  // dw[r][c] += acc for c < K; db[r] += acc for c == K
    float *dw, *db;
    int rows, K;
    __device__ void operator()(int r, int c, float v) const {
        if (r >= rows || c > K) return;
        if (c < K) atomicAdd(&dw[(size_t)r * K + c], v);
        else if (db) atomicAdd(&db[r], v);
    }
};

// C[rows][cols] = sum over the reduction range [z * ksplit, min(Kred, (z + 1) * ksplit))
// of A(row, k) B(col, k); block tile 128 x 64 x 32, 8 warps of 32 x 32.
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(GT) k_gemm(LA la, LB lb, EP ep, int Kred, int ksplit) {
    __shared__ __align__(16) bf16 sA[2][BM * LDS];
    __shared__ __align__(16) bf16 sB[2][BN * LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * ksplit, ke = min(Kred, kb + ksplit);
    if (kb >= ke) return;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    uint4 ra0, ra1, rb0;
    auto load = [&](int k) {
        ra0 = la(m0 + (tid >> 2), k + (tid & 3) * 8, ke);
        ra1 = la(m0 + 64 + (tid >> 2), k + (tid & 3) * 8, ke);
        rb0 = lb(n0 + (tid >> 2), k + (tid & 3) * 8, ke);
    };
    auto store = [&](int buf) {
        *reinterpret_cast<uint4 *>(&sA[buf][(tid >> 2) * LDS + (tid & 3) * 8]) = ra0;
        *reinterpret_cast<uint4 *>(&sA[buf][(64 + (tid >> 2)) * LDS + (tid & 3) * 8]) = ra1;
        *reinterpret_cast<uint4 *>(&sB[buf][(tid >> 2) * LDS + (tid & 3) * 8]) = rb0;
    };
    load(kb);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k = kb; k < ke; k += BK) {
        const bool more = k + BK < ke;
        if (more) load(k + BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                ldsm_x4(a[i], &sA[buf][r * LDS + kk + (lane >> 4) * 8]);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r = wn * 32 + j * 16 + (lane & 7) + (lane >> 4) * 8;
                uint32_t t[4];
                ldsm_x4(t, &sB[buf][r * LDS + kk + ((lane >> 3) & 1) * 8]);
                b[2 * j][0] = t[0];
                b[2 * j][1] = t[1];
                b[2 * j + 1][0] = t[2];
                b[2 * j + 1][1] = t[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
        }
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + wm * 32 + i * 16 + (lane >> 2);
            const int c = n0 + wn * 32 + j * 8 + (lane & 3) * 2;
            ep(r, c, acc[i][j][0]);
            ep(r, c + 1, acc[i][j][1]);
            ep(r + 8, c, acc[i][j][2]);
            ep(r + 8, c + 1, acc[i][j][3]);
        }
}

template <class LA, class LB, class EP>
cudaError_t gemm(LA la, LB lb, EP ep, int rows, int cols, int Kred, int ksplit, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || Kred <= 0) return cudaSuccess;
    ksplit = std::max(BK, (ksplit + BK - 1) / BK * BK);
    const dim3 grid((rows + BM - 1) / BM, (cols + BN - 1) / BN, (Kred + ksplit - 1) / ksplit);
    if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidValue;
    k_gemm<LA, LB, EP><<<grid, GT, 0, st>>>(la, lb, ep, Kred, ksplit);
    return cudaGetLastError();
}

// ------------------------------------------------------- element kernels
// dx[b][ih][iw][ci] = sum over the (kh, kw) taps whose output position exists of
// D[(b, oh, ow)][(kh, kw, ci)], times (mask > 0) when given.
__global__ void k_col2im(const float *__restrict__ dcol, ConvShape s, const bf16 *__restrict__ mask,
                         bf16 *__restrict__ dx, float *__restrict__ dx32) {
    const int64_t n = (int64_t)s.B * s.H * s.W * s.Ci;
    const int K9 = 9 * s.Ci;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(e % s.Ci);
        int64_t t = e / s.Ci;
        const int iw = (int)(t % s.W);
        t /= s.W;
        const int ih = (int)(t % s.H);
        const int b = (int)(t / s.H);
        float v = 0.f;
#pragma unroll
        for (int kh = 0; kh < 3; ++kh) {
            const int y2 = ih + 1 - kh;
            if (y2 < 0 || (y2 & 1) || (y2 >> 1) >= s.OH) continue;
#pragma unroll
            for (int kw = 0; kw < 3; ++kw) {
                const int x2 = iw + 1 - kw;
                if (x2 < 0 || (x2 & 1) || (x2 >> 1) >= s.OW) continue;
                const int64_t m = ((int64_t)b * s.OH + (y2 >> 1)) * s.OW + (x2 >> 1);
                v += dcol[m * K9 + (kh * 3 + kw) * s.Ci + ci];
            }
        }
        if (mask && !(__bfloat162float(mask[e]) > 0.f)) v = 0.f;
        dx[e] = __float2bfloat16(v);
        if (dx32) dx32[e] = v;
    }
}

// Weights [Co][K] -> transposed [K][Co].
__global__ void k_transpose_bf16(const bf16 *__restrict__ w, int Co, int K, bf16 *__restrict__ wt) {
    __shared__ bf16 tile[32][33];
    const int k0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, k = k0 + threadIdx.x;
        if (c < Co && k < K) tile[r][threadIdx.x] = w[(size_t)c * K + k];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, c = c0 + threadIdx.x;
        if (c < Co && k < K) wt[(size_t)k * Co + c] = tile[threadIdx.x][r];
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, int64_t n, bf16 *__restrict__ b) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = __float2bfloat16(a[e]);
}

// First layer (one input channel, 32 outputs): a thread per output position.
__global__ void k_conv1_fwd(const bf16 *__restrict__ x, ConvShape s, const bf16 *__restrict__ w,
                            const float *__restrict__ bias, bf16 *__restrict__ y) {
    __shared__ float ws[32 * 9], bs[32];
    for (int e = threadIdx.x; e < 32 * 9; e += blockDim.x) ws[e] = __bfloat162float(w[e]);
    for (int e = threadIdx.x; e < 32; e += blockDim.x) bs[e] = bias[e];
    __syncthreads();
    const int64_t M = (int64_t)s.B * s.OH * s.OW;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const int ow = (int)(m % s.OW);
        const int64_t t = m / s.OW;
        const int oh = (int)(t % s.OH), b = (int)(t / s.OH);
        float xv[9];
#pragma unroll
        for (int kh = 0; kh < 3; ++kh)
#pragma unroll
            for (int kw = 0; kw < 3; ++kw) {
                const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
                xv[kh * 3 + kw] = (ih >= 0 && ih < s.H && iw >= 0 && iw < s.W)
                                      ? __bfloat162float(x[((size_t)b * s.H + ih) * s.W + iw])
                                      : 0.f;
            }
        bf16 out[32];
#pragma unroll
        for (int co = 0; co < 32; ++co) {
            float v = bs[co];
#pragma unroll
            for (int k = 0; k < 9; ++k) v = fmaf(ws[co * 9 + k], xv[k], v);
            out[co] = __float2bfloat16(fmaxf(v, 0.f));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)m * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = pack8(out + 8 * q);
    }
}

// First-layer weight gradient: lane = output channel, warps stride over positions.
__global__ void __launch_bounds__(256) k_conv1_wgrad(const bf16 *__restrict__ g, const bf16 *__restrict__ x,
                                                     ConvShape s, float *__restrict__ dw, float *__restrict__ db) {
    __shared__ float red[8][32][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int64_t M = (int64_t)s.B * s.OH * s.OW;
    for (int64_t m = (int64_t)blockIdx.x * 8 + warp; m < M; m += (int64_t)gridDim.x * 8) {
        const int ow = (int)(m % s.OW);
        const int64_t t = m / s.OW;
        const int oh = (int)(t % s.OH), b = (int)(t / s.OH);
        const float gv = __bfloat162float(g[m * 32 + lane]);
#pragma unroll
        for (int kh = 0; kh < 3; ++kh)
#pragma unroll
            for (int kw = 0; kw < 3; ++kw) {
                const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
                const float xv = (ih >= 0 && ih < s.H && iw >= 0 && iw < s.W)
                                     ? __bfloat162float(x[((size_t)b * s.H + ih) * s.W + iw])
                                     : 0.f;
                acc[kh * 3 + kw] = fmaf(gv, xv, acc[kh * 3 + kw]);
            }
        acc[9] += gv;
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) red[warp][lane][k] = acc[k];
    __syncthreads();
    for (int e = threadIdx.x; e < 320; e += blockDim.x) {
        const int co = e / 10, k = e - 10 * co;
        float v = 0.f;
        for (int ww = 0; ww < 8; ++ww) v += red[ww][co][k];
        if (k < 9) atomicAdd(&dw[co * 9 + k], v);
        else atomicAdd(&db[co], v);
    }
}

// ------------------------------------------------------------ float32 head
// h[b] = (y[b] flattened position-major (p, c), aux[b]).
__global__ void k_flatten_concat(const bf16 *__restrict__ y, int B, int F, const float *__restrict__ aux,
                                 float *__restrict__ h) {
    const int HD = F + kAux;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * HD; e += gridDim.x * blockDim.x) {
        const int b = e / HD, c = e - b * HD;
        h[e] = c < F ? __bfloat162float(y[(size_t)b * F + c]) : aux[b * kAux + (c - F)];
    }
}
// out[b][j] = bias[j] + sum_i W[j][i] in[b][i], optionally ReLU (z keeps the pre-activation).
__global__ void k_fc(const float *__restrict__ in, int B, int I, const float *__restrict__ W,
                     const float *__restrict__ bias, int J, int relu, float *__restrict__ z, float *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * J; e += gridDim.x * blockDim.x) {
        const int b = e / J, j = e - b * J;
        float v = bias[j];
        const float *wr = W + (size_t)j * I, *xr = in + (size_t)b * I;
        for (int i = 0; i < I; ++i) v = fmaf(wr[i], xr[i], v);
        if (z) z[e] = v;
        out[e] = relu ? fmaxf(v, 0.f) : v;
    }
}
// d = 2 (out - target) / (6 B); loss = mean squared error (one block).
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ tgt, int n, float *__restrict__ d,
                      double *loss) {
    __shared__ double red[256];
    double s = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const float r = out[e] - tgt[e];
        d[e] = 2.f * r / (float)n;
        s += (double)r * r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = red[0] / (double)n;
}
// dW[j][i] = sum_b d[b][j] in[b][i]; db[j] = sum_b d[b][j].
__global__ void k_fc_wgrad(const float *__restrict__ d, const float *__restrict__ in, int B, int I, int J,
                           float *__restrict__ dW, float *__restrict__ db) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J * (I + 1); e += gridDim.x * blockDim.x) {
        const int j = e / (I + 1), i = e - j * (I + 1);
        float v = 0.f;
        if (i < I)
            for (int b = 0; b < B; ++b) v = fmaf(d[b * J + j], in[(size_t)b * I + i], v);
        else
            for (int b = 0; b < B; ++b) v += d[b * J + j];
        if (i < I) dW[(size_t)j * I + i] = v;
        else db[j] = v;
    }
}
// din[b][i] = sum_j d[b][j] W[j][i], times (zin > 0) when zin is given.
__global__ void k_fc_dgrad(const float *__restrict__ d, const float *__restrict__ W, int B, int I, int J,
                           const float *__restrict__ zin, float *__restrict__ din) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * I; e += gridDim.x * blockDim.x) {
        const int b = e / I, i = e - b * I;
        float v = 0.f;
        for (int j = 0; j < J; ++j) v = fmaf(d[b * J + j], W[(size_t)j * I + i], v);
        if (zin && !(zin[e] > 0.f)) v = 0.f;
        din[e] = v;
    }
}
// g[b][f] = dh[b][f] times (y > 0) over the flattened features; bfloat16.
__global__ void k_flatten_grad(const float *__restrict__ dh, int B, int F, int HD, const bf16 *__restrict__ y,
                               bf16 *__restrict__ g) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * F; e += gridDim.x * blockDim.x) {
        const int b = e / F, f = e - b * F;
        g[e] = __float2bfloat16(__bfloat162float(y[e]) > 0.f ? dh[b * HD + f] : 0.f);
    }
}
__global__ void k_adam_flat(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float ibc1,
                            float ibc2) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi * ibc1) / (sqrtf(vi * ibc2) + eps);
    }
}

int blocks_for(int64_t n, int per = 256) { return (int)std::min<int64_t>((n + per - 1) / per, 148 * 16); }

ConvShape conv_shape(int B, int H, int W, int Ci, int Co) { return ConvShape{B, H, W, Ci, (H + 1) / 2, (W + 1) / 2, Co}; }

// --------------------------------------------------------- conv operations
cudaError_t conv_forward(const bf16 *x, const ConvShape &s, const bf16 *w, const float *bias, int relu, bf16 *y,
                         float *y32, cudaStream_t st) {
    const int M = s.B * s.OH * s.OW, K = 9 * s.Ci;
    if (s.Ci == 1 && s.Co == 32 && relu && !y32) {
        k_conv1_fwd<<<blocks_for(M), 256, 0, st>>>(x, s, w, bias, y);
        return cudaGetLastError();
    }
    return gemm(LoadIm2col{x, s, M, K}, LoadRows{w, s.Co, K}, EpiConv{y, y32, bias, M, s.Co, relu}, M, s.Co, K, K,
                st);
}

cudaError_t conv_dgrad(const bf16 *gy, const ConvShape &s, const bf16 *w, bf16 *wt, const bf16 *mask, float *dcol,
                       bf16 *dx, float *dx32, cudaStream_t st) {
    const int M = s.B * s.OH * s.OW, K = 9 * s.Ci;
    k_transpose_bf16<<<dim3((K + 31) / 32, (s.Co + 31) / 32), dim3(32, 8), 0, st>>>(w, s.Co, K, wt);
    cudaError_t e = gemm(LoadRows{gy, M, s.Co}, LoadRows{wt, K, s.Co}, EpiStore{dcol, M, K, K}, M, K, s.Co, s.Co, st);
    if (e != cudaSuccess) return e;
    k_col2im<<<blocks_for((int64_t)s.B * s.H * s.W * s.Ci), 256, 0, st>>>(dcol, s, mask, dx, dx32);
    return cudaGetLastError();
}

cudaError_t conv_wgrad(const bf16 *gy, const bf16 *x, const ConvShape &s, float *dw, float *db, cudaStream_t st) {
    const int M = s.B * s.OH * s.OW, K = 9 * s.Ci;
    if (s.Ci == 1 && s.Co == 32) {
        k_conv1_wgrad<<<std::min(std::max(1, M / 64), 148 * 8), 256, 0, st>>>(gy, x, s, dw, db);
        return cudaGetLastError();
    }
    // reduction over positions split so that the grid fills the GPU a few times
    const int tiles = ((s.Co + BM - 1) / BM) * ((K + 1 + BN - 1) / BN);
    const int splits = std::max(1, std::min((M + BK - 1) / BK, (148 * 4 + tiles - 1) / tiles));
    const int ksplit = (M + splits - 1) / splits;
    return gemm(LoadCols{gy, s.Co, s.Co}, LoadIm2colT{x, s, K}, EpiWgrad{dw, db, s.Co, K}, s.Co, K + 1, M, ksplit,
                st);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

thread_local std::string g_cnn_error;

}  // namespace

// ------------------------------------------------------------------- model
struct gsvr_cnn {
    int device = 0;
    cudaStream_t st = nullptr;
    int max_batch = 0;
    std::string err;
    int64_t n_params = 0;
    int64_t off_w[kLayers], off_b[kLayers], off_fc1w, off_fc1b, off_fc2w, off_fc2b;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wbf = nullptr;   // bfloat16 copy of the whole parameter vector (conv weights used)
    bf16 *wt = nullptr;    // transposed weights scratch
    bf16 *act[kLayers + 1] = {};
    bf16 *gpre[kLayers + 1] = {};  // gradient at each conv output (after the ReLU mask)
    float *dcol = nullptr;
    float *h = nullptr, *z1 = nullptr, *a1 = nullptr, *out = nullptr, *dout = nullptr, *dz1 = nullptr, *dh = nullptr;
    std::vector<void *> allocs;
    ~gsvr_cnn() {
        for (void *p : allocs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T *&p, size_t n) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        p = static_cast<T *>(q);
        return cudaSuccess;
    }
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

gsvr_status nfail(gsvr_cnn *n, gsvr_status s, const std::string &msg) {
    if (n) n->err = msg;
    else g_cnn_error = msg;
    return s;
}
gsvr_status cuda_status(gsvr_cnn *n, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GSVR_OK;
    cudaGetLastError();
    return nfail(n, e == cudaErrorMemoryAllocation ? GSVR_ERR_NOMEM : GSVR_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

int layer_size(int l) { return kImage >> l; }  // spatial side of act[l]

gsvr_status run_forward(gsvr_cnn *n, const float *x, const float *aux, int B) {
    cudaStream_t st = n->st;
    k_to_bf16<<<blocks_for(n->n_params), 256, 0, st>>>(n->params, n->n_params, n->wbf);
    k_to_bf16<<<blocks_for((int64_t)B * kImage * kImage), 256, 0, st>>>(x, (int64_t)B * kImage * kImage, n->act[0]);
    for (int l = 0; l < kLayers; ++l) {
        const ConvShape s = conv_shape(B, layer_size(l), layer_size(l), kCh[l], kCh[l + 1]);
        cudaError_t e = conv_forward(n->act[l], s, n->wbf + n->off_w[l], n->params + n->off_b[l], 1, n->act[l + 1],
                                     nullptr, st);
        if (e != cudaSuccess) return cuda_status(n, e, "conv forward");
    }
    const int F = layer_size(kLayers) * layer_size(kLayers) * kCh[kLayers], HD = F + kAux;
    k_flatten_concat<<<blocks_for((int64_t)B * HD), 256, 0, st>>>(n->act[kLayers], B, F, aux, n->h);
    k_fc<<<blocks_for((int64_t)B * kHidden), 256, 0, st>>>(n->h, B, HD, n->params + n->off_fc1w,
                                                           n->params + n->off_fc1b, kHidden, 1, n->z1, n->a1);
    k_fc<<<blocks_for((int64_t)B * kOut), 256, 0, st>>>(n->a1, B, kHidden, n->params + n->off_fc2w,
                                                        n->params + n->off_fc2b, kOut, 0, nullptr, n->out);
    return cuda_status(n, cudaGetLastError(), "head forward");
}

}  // namespace

extern "C" {

gsvr_status gsvr_cnn_create(gsvr_cnn **out, int32_t device, void *stream, int32_t max_batch, uint64_t seed) {
    g_cnn_error.clear();
    if (!out || max_batch < 1 || max_batch > 4096) return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad arguments");
    *out = nullptr;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) {
        cudaGetLastError();
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "no such CUDA device");
    }
    DevGuard g(device);
    gsvr_cnn *n = new (std::nothrow) gsvr_cnn();
    if (!n) return nfail(nullptr, GSVR_ERR_NOMEM, "host allocation failed");
    n->device = device;
    n->st = static_cast<cudaStream_t>(stream);
    n->max_batch = max_batch;
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        n->off_w[l] = o;
        o += (int64_t)kCh[l + 1] * 9 * kCh[l];
        n->off_b[l] = o;
        o += kCh[l + 1];
    }
    const int HD = layer_size(kLayers) * layer_size(kLayers) * kCh[kLayers] + kAux;
    n->off_fc1w = o;
    o += (int64_t)kHidden * HD;
    n->off_fc1b = o;
    o += kHidden;
    n->off_fc2w = o;
    o += (int64_t)kOut * kHidden;
    n->off_fc2b = o;
    o += kOut;
    n->n_params = o;
    // He-normal weights, zero biases
    std::vector<float> p((size_t)o, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int64_t off, int64_t cnt, int fan_in) {
        std::normal_distribution<double> nd2(0.0, std::sqrt(2.0 / fan_in));
        for (int64_t k = 0; k < cnt; ++k) p[(size_t)(off + k)] = (float)nd2(rng);
    };
    for (int l = 0; l < kLayers; ++l) fill(n->off_w[l], (int64_t)kCh[l + 1] * 9 * kCh[l], 9 * kCh[l]);
    fill(n->off_fc1w, (int64_t)kHidden * HD, HD);
    fill(n->off_fc2w, (int64_t)kOut * kHidden, kHidden);
    cudaError_t e = cudaSuccess;
    const int B = max_batch;
    size_t dcol_max = 0, wt_max = 0;
    for (int l = 1; l < kLayers; ++l) {
        const size_t M = (size_t)B * layer_size(l + 1) * layer_size(l + 1);
        dcol_max = std::max(dcol_max, M * 9 * kCh[l]);
        wt_max = std::max(wt_max, (size_t)9 * kCh[l] * kCh[l + 1]);
    }
    if (!e) e = n->alloc(n->params, o);
    if (!e) e = n->alloc(n->grads, o);
    if (!e) e = n->alloc(n->m, o);
    if (!e) e = n->alloc(n->v, o);
    if (!e) e = n->alloc(n->wbf, o);
    if (!e) e = n->alloc(n->wt, wt_max);
    for (int l = 0; l <= kLayers && !e; ++l) {
        const size_t sz = (size_t)B * layer_size(l) * layer_size(l) * kCh[l];
        e = n->alloc(n->act[l], sz);
        if (!e) e = n->alloc(n->gpre[l], sz);
    }
    if (!e) e = n->alloc(n->dcol, dcol_max);
    if (!e) e = n->alloc(n->h, (size_t)B * HD);
    if (!e) e = n->alloc(n->z1, (size_t)B * kHidden);
    if (!e) e = n->alloc(n->a1, (size_t)B * kHidden);
    if (!e) e = n->alloc(n->out, (size_t)B * kOut);
    if (!e) e = n->alloc(n->dout, (size_t)B * kOut);
    if (!e) e = n->alloc(n->dz1, (size_t)B * kHidden);
    if (!e) e = n->alloc(n->dh, (size_t)B * HD);
    if (!e) e = cudaMemcpy(n->params, p.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(n->grads, 0, sizeof(float) * o);
    if (!e) e = cudaMemset(n->m, 0, sizeof(float) * o);
    if (!e) e = cudaMemset(n->v, 0, sizeof(float) * o);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_cnn_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
        delete n;
        return e == cudaErrorMemoryAllocation ? GSVR_ERR_NOMEM : GSVR_ERR_CUDA;
    }
    *out = n;
    return GSVR_OK;
}

gsvr_status gsvr_cnn_destroy(gsvr_cnn *n) {
    if (!n) return GSVR_ERR_INVALID_ARG;
    DevGuard g(n->device);
    cudaStreamSynchronize(n->st);
    cudaGetLastError();
    delete n;
    return GSVR_OK;
}

const char *gsvr_cnn_last_error(gsvr_cnn *n) { return n ? n->err.c_str() : g_cnn_error.c_str(); }

gsvr_status gsvr_cnn_views(gsvr_cnn *n, float **params, float **grads, int64_t *n_params) {
    if (!n) return GSVR_ERR_INVALID_ARG;
    if (params) *params = n->params;
    if (grads) *grads = n->grads;
    if (n_params) *n_params = n->n_params;
    return GSVR_OK;
}

gsvr_status gsvr_cnn_forward(gsvr_cnn *n, const float *x, const float *aux, int32_t B, float *out) {
    if (!n) return GSVR_ERR_INVALID_ARG;
    if (!x || !aux || !out || B < 1 || B > n->max_batch)
        return nfail(n, GSVR_ERR_INVALID_ARG, "need x, aux, out and 1 <= B <= max_batch");
    DevGuard g(n->device);
    gsvr_status s = run_forward(n, x, aux, B);
    if (s) return s;
    return cuda_status(n, cudaMemcpyAsync(out, n->out, sizeof(float) * B * kOut, cudaMemcpyDeviceToDevice, n->st),
                       "copy out");
}

gsvr_status gsvr_cnn_loss_backward(gsvr_cnn *n, const float *x, const float *aux, const float *target, int32_t B,
                                   double *loss) {
    if (!n) return GSVR_ERR_INVALID_ARG;
    if (!x || !aux || !target || B < 1 || B > n->max_batch)
        return nfail(n, GSVR_ERR_INVALID_ARG, "need x, aux, target and 1 <= B <= max_batch");
    DevGuard g(n->device);
    cudaStream_t st = n->st;
    gsvr_status s = run_forward(n, x, aux, B);
    if (s) return s;
    const int F = layer_size(kLayers) * layer_size(kLayers) * kCh[kLayers], HD = F + kAux;
    cudaError_t e = cudaMemsetAsync(n->grads, 0, sizeof(float) * n->n_params, st);
    if (e) return cuda_status(n, e, "zero gradients");
    k_mse<<<1, 256, 0, st>>>(n->out, target, B * kOut, n->dout, loss);
    k_fc_wgrad<<<blocks_for((int64_t)kOut * (kHidden + 1)), 256, 0, st>>>(
        n->dout, n->a1, B, kHidden, kOut, n->grads + n->off_fc2w, n->grads + n->off_fc2b);
    k_fc_dgrad<<<blocks_for((int64_t)B * kHidden), 256, 0, st>>>(n->dout, n->params + n->off_fc2w, B, kHidden, kOut,
                                                                 n->z1, n->dz1);
    k_fc_wgrad<<<blocks_for((int64_t)kHidden * (HD + 1)), 256, 0, st>>>(
        n->dz1, n->h, B, HD, kHidden, n->grads + n->off_fc1w, n->grads + n->off_fc1b);
    k_fc_dgrad<<<blocks_for((int64_t)B * HD), 256, 0, st>>>(n->dz1, n->params + n->off_fc1w, B, HD, kHidden, nullptr,
                                                            n->dh);
    k_flatten_grad<<<blocks_for((int64_t)B * F), 256, 0, st>>>(n->dh, B, F, HD, n->act[kLayers],
                                                               n->gpre[kLayers]);
    e = cudaGetLastError();
    if (e) return cuda_status(n, e, "head backward");
    for (int l = kLayers - 1; l >= 0; --l) {
        const ConvShape sh = conv_shape(B, layer_size(l), layer_size(l), kCh[l], kCh[l + 1]);
        e = conv_wgrad(n->gpre[l + 1], n->act[l], sh, n->grads + n->off_w[l], n->grads + n->off_b[l], st);
        if (e) return cuda_status(n, e, "conv wgrad");
        if (l > 0) {
            e = conv_dgrad(n->gpre[l + 1], sh, n->wbf + n->off_w[l], n->wt, n->act[l], n->dcol, n->gpre[l], nullptr,
                           st);
            if (e) return cuda_status(n, e, "conv dgrad");
        }
    }
    return GSVR_OK;
}

gsvr_status gsvr_cnn_adam_step(gsvr_cnn *n, float lr, float beta1, float beta2, float eps, int64_t t) {
    if (!n) return GSVR_ERR_INVALID_ARG;
    const float b1 = beta1 == 0.f ? 0.9f : beta1, b2 = beta2 == 0.f ? 0.999f : beta2, ep = eps == 0.f ? 1e-8f : eps;
    if (t < 1 || !(lr >= 0.f) || !(b1 > 0.f && b1 < 1.f && b2 > 0.f && b2 < 1.f && ep > 0.f))
        return nfail(n, GSVR_ERR_INVALID_ARG, "bad Adam arguments");
    DevGuard g(n->device);
    const float ibc1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)t)));
    const float ibc2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)t)));
    k_adam_flat<<<blocks_for(n->n_params), 256, 0, n->st>>>(n->params, n->grads, n->m, n->v, n->n_params, lr, b1, b2,
                                                            ep, ibc1, ibc2);
    return cuda_status(n, cudaGetLastError(), "adam");
}

gsvr_status gsvr_cnn_conv_forward(void *stream, const uint16_t *x, int32_t B, int32_t H, int32_t W, int32_t Ci,
                                  const uint16_t *w, const float *bias, int32_t Co, int32_t relu, uint16_t *y,
                                  float *y32) {
    g_cnn_error.clear();
    if (!x || !w || !y || B < 1 || H < 1 || W < 1 || Ci < 1 || Co < 2 || (Co & 1) || (Ci % 8 && Ci != 1) ||
        !aligned16(x) || !aligned16(w) || (int64_t)B * H * W > (1LL << 30))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad conv forward arguments");
    const ConvShape s = conv_shape(B, H, W, Ci, Co);
    if (Ci == 1 && !(Co == 32 && relu && !y32 && bias))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "one input channel: Co 32, ReLU, bias, no y32");
    return cuda_status(nullptr,
                       conv_forward(reinterpret_cast<const bf16 *>(x), s, reinterpret_cast<const bf16 *>(w), bias, relu,
                                    reinterpret_cast<bf16 *>(y), y32, static_cast<cudaStream_t>(stream)),
                       "conv forward");
}

gsvr_status gsvr_cnn_conv_dgrad(void *stream, const uint16_t *gy, int32_t B, int32_t H, int32_t W, int32_t Ci,
                                const uint16_t *w, int32_t Co, const uint16_t *mask, float *dcol, uint16_t *dx,
                                float *dx32) {
    g_cnn_error.clear();
    if (!gy || !w || !dcol || !dx || B < 1 || H < 1 || W < 1 || Ci < 8 || (Ci % 8) || Co < 8 || (Co % 8) ||
        !aligned16(gy) || !aligned16(w) || (int64_t)B * H * W > (1LL << 30))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad conv dgrad arguments (Ci, Co multiples of 8)");
    const ConvShape s = conv_shape(B, H, W, Ci, Co);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bf16 *wt = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&wt), sizeof(bf16) * 9 * Ci * Co, st);
    if (e) return cuda_status(nullptr, e, "scratch");
    e = conv_dgrad(reinterpret_cast<const bf16 *>(gy), s, reinterpret_cast<const bf16 *>(w), wt,
                   reinterpret_cast<const bf16 *>(mask), dcol, reinterpret_cast<bf16 *>(dx), dx32, st);
    cudaFreeAsync(wt, st);
    return cuda_status(nullptr, e, "conv dgrad");
}

gsvr_status gsvr_cnn_conv_wgrad(void *stream, const uint16_t *gy, const uint16_t *x, int32_t B, int32_t H, int32_t W,
                                int32_t Ci, int32_t Co, float *dw, float *db) {
    g_cnn_error.clear();
    if (!gy || !x || !dw || B < 1 || H < 1 || W < 1 || Ci < 1 || (Ci % 8 && Ci != 1) || Co < 2 || (Co & 1) ||
        (Ci == 1 && (Co != 32 || !db)) || (int64_t)B * H * W > (1LL << 30))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad conv wgrad arguments");
    const ConvShape s = conv_shape(B, H, W, Ci, Co);
    return cuda_status(nullptr,
                       conv_wgrad(reinterpret_cast<const bf16 *>(gy), reinterpret_cast<const bf16 *>(x), s, dw, db,
                                  static_cast<cudaStream_t>(stream)),
                       "conv wgrad");
}

}  // extern "C"
