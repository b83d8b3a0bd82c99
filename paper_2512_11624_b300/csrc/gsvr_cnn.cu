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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <vector>

#include "gsvr_cnn.h"
#include "gsvr_internal.cuh"

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
// two floats rounded to bfloat16, lo in the low half
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
struct ConvShape {
    int B, H, W, Ci, OH, OW, Co;
    int lOW, lOH, lCi, lCo;  // log2 of OW, OH, Ci, Co when a power of two, else -1
};

// m = (b, oh, ow) -> its parts (shifts when the sides are powers of two)
__device__ __forceinline__ void pos_split(const ConvShape &s, int m, int &b, int &oh, int &ow) {
    int t;
    if (s.lOW >= 0) {
        ow = m & (s.OW - 1);
        t = m >> s.lOW;
    } else {
        t = m / s.OW;
        ow = m - t * s.OW;
    }
    if (s.lOH >= 0) {
        oh = t & (s.OH - 1);
        b = t >> s.lOH;
    } else {
        b = t / s.OH;
        oh = t - b * s.OH;
    }
}
// k = (q, c) over C channels -> q, c
__device__ __forceinline__ void chan_split(int k, int C, int lC, int &q, int &c) {
    if (lC >= 0) {
        q = k >> lC;
        c = k & (C - 1);
    } else {
        q = k / C;
        c = k - q * C;
    }
}

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
        int tap, ci, b, oh, ow;
        chan_split(k0, s.Ci, s.lCi, tap, ci);
        const int kh = (tap * 11) >> 5, kw = tap - 3 * kh;  // tap / 3 for tap < 9
        pos_split(s, m, b, oh, ow);
        const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
        if (ih < 0 || ih >= s.H || iw < 0 || iw >= s.W) return zero4();
        return *reinterpret_cast<const uint4 *>(x + (((size_t)b * s.H + ih) * s.W + iw) * s.Ci + ci);
    }
    // address of the same 8 values, nullptr where they are zero (padding, past the ends)
    __device__ const bf16 *src(int m, int k0, int k_end) const {
        if (m >= rows || k0 >= k_end) return nullptr;
        int tap, ci, b, oh, ow;
        chan_split(k0, s.Ci, s.lCi, tap, ci);
        const int kh = (tap * 11) >> 5, kw = tap - 3 * kh;
        pos_split(s, m, b, oh, ow);
        const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
        if (ih < 0 || ih >= s.H || iw < 0 || iw >= s.W) return nullptr;
        return x + (((size_t)b * s.H + ih) * s.W + iw) * s.Ci + ci;
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
    __device__ const bf16 *src(int r, int k0, int k_end) const {
        return (r >= rows || k0 >= k_end) ? nullptr : p + (size_t)r * ld + k0;
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
    // columns c0 .. c0 + 7 of row r (c0 % 8 == 0)
    __device__ void vec8(int r, int c0, const float *v) const {
        if (r >= rows) return;
        if (c0 + 8 > cols || (cols & 7)) {
            for (int j = 0; j < 8; ++j) (*this)(r, c0 + j, v[j]);
            return;
        }
        float o[8];
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            o[j] = v[j] + (bias ? bias[c0 + j] : 0.f);
            if (relu) o[j] = fmaxf(o[j], 0.f);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) pk[j] = pack_bf16x2(o[2 * j], o[2 * j + 1]);
        const size_t e = (size_t)r * cols + c0;
        *reinterpret_cast<uint4 *>(y + e) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        if (y32) {
            reinterpret_cast<float4 *>(y32 + e)[0] = make_float4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<float4 *>(y32 + e)[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
    }
    // columns c0 .. c0 + 31 (c0 % 32 == 0): the bias is read before any store
    __device__ void vec32(int r, int c0, const float *v) const {
        if (r >= rows) return;
        if (c0 + 32 > cols || (cols & 7) || !bias) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) vec8(r, c0 + j, v + j);
            return;
        }
        float o[32];
        const float4 *b4 = reinterpret_cast<const float4 *>(bias + c0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 b = __ldg(b4 + j);
            o[4 * j] = v[4 * j] + b.x;
            o[4 * j + 1] = v[4 * j + 1] + b.y;
            o[4 * j + 2] = v[4 * j + 2] + b.z;
            o[4 * j + 3] = v[4 * j + 3] + b.w;
        }
        if (relu) {
#pragma unroll
            for (int j = 0; j < 32; ++j) o[j] = fmaxf(o[j], 0.f);
        }
        const size_t e = (size_t)r * cols + c0;
#pragma unroll
        for (int g = 0; g < 4; ++g)
            reinterpret_cast<uint4 *>(y + e)[g] =
                make_uint4(pack_bf16x2(o[8 * g], o[8 * g + 1]), pack_bf16x2(o[8 * g + 2], o[8 * g + 3]),
                           pack_bf16x2(o[8 * g + 4], o[8 * g + 5]), pack_bf16x2(o[8 * g + 6], o[8 * g + 7]));
        if (y32) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                reinterpret_cast<float4 *>(y32 + e)[j] = make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
        }
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

// ------------------------------------------------ 5th-generation tensor cores
// tcgen05 GEMM: C[rows][cols] = sum_k A(row, k) B(col, k) with bfloat16 operands
// and float32 accumulators in tensor memory.  A CTA of 128 threads owns a
// Output tile 128 x BN (BN = 64 or 128) accumulated in tensor memory, warp
// specialised.  Warps 0-3 produce: per 64-wide K step they copy both operand
// tiles from global memory with 16-byte cp.async (zero-filled where the loader
// reports padding) into shared memory in the 128-byte-swizzled K-major layout
// (8-row x 128-byte atoms, 16-byte chunk c of row r at r * 128 +
// ((c ^ (r % 8)) * 16), atoms 1024 bytes apart); each thread signals a stage's
// `full` barrier TC_LAG steps later, once its copies have landed and are
// fenced for the tensor cores.  Warp 4 owns the tensor memory: one thread
// waits for `full`, issues the four tcgen05.mma (K = 16 each) of the step and
// commits them to the stage's `empty` barrier, which frees the stage for the
// producers.  STAGES steps are resident; no CTA-wide barrier runs per step.
// After the last step warps 0-3 read the accumulators back with tcgen05.ld
// (warp w owns rows 32 w .. 32 w + 31, 32 columns per load) and store 8
// columns at a time.
constexpr int TC_M = 128, TC_K = 64, TC_PRODUCERS = 128, TC_THREADS = TC_PRODUCERS + 32, TC_LAG = 2;
constexpr uint64_t kTcWaitNs = 1000000000ull;  // 1 s bound on every mbarrier wait
template <int BN>
struct TcCfg {
    static constexpr int STAGES = BN == 128 ? 3 : 4;  // two CTAs per SM either way
    static constexpr int A_BYTES = TC_M * TC_K * 2, B_BYTES = BN * TC_K * 2, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;  // + alignment slack
    // instruction descriptor, kind::f16: D float32 (bits 4-5 = 1), A and B
    // bfloat16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(TC_M >> 4) << 24);
    static_assert(TC_LAG < STAGES, "a producer must signal a stage before it waits to refill it");
};

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
    // matrix descriptor: start >> 4 [0,14), leading byte offset >> 4 [16,30)
    // (unused by swizzled K-major layouts: 1), stride byte offset >> 4 [32,46)
    // (1024 B between 8-row atoms), fixed 0b001 at [46,49), swizzle 128 B (2) at [61,64)
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// K-major, 64-byte swizzle: 8-row x 64-byte atoms 512 bytes apart, swizzle mode 4
__device__ __forceinline__ uint64_t tc_smem_desc64(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(512u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)4u << 61);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     gsvr::smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared; src == nullptr writes zeros
// (source size 0: nothing is read, the base pointer only stands in).
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, const void *base) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src ? src : base),
                 "r"(src ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gsvr::smem_u32(bar)) : "memory");
}

template <class LA, class LB, class EP, int BN>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(LA la, LB lb, EP ep, int Kred, const void *base,
                                                        unsigned *status) {
    using Cfg = TcCfg<BN>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * BN;
    const uint32_t sbase = (gsvr::smem_u32(tc_raw) + 1023u) & ~1023u;
    const int nk = (Kred + TC_K - 1) / TC_K;
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gsvr::smem_u32(&s_tmem)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            gsvr::mbar_init(&full[i], TC_PRODUCERS);
            gsvr::mbar_init(&empty[i], 1);
        }
        gsvr::mbar_init(&done, 1);
        gsvr::fence_mbar_init();
        s_fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (warp < 4) {
        // ---- producers: step kt into stage kt % S; signal step kt - TC_LAG
        auto signal = [&](int j) {
            cp_async_wait_group<TC_LAG>();  // this thread's copies of step j have landed
            gsvr::fence_proxy_async_smem();  // ... and are visible to the tensor cores
            mbar_arrive(&full[j % S]);
        };
        for (int kt = 0; kt < nk + TC_LAG; ++kt) {
            if (kt < nk) {
                const int s = kt % S;
                if (kt >= S && !gsvr::mbar_wait_bounded(&empty[s], ((kt / S) - 1) & 1u, kTcWaitNs)) s_fail = 1;
                if (s_fail) break;
                const uint32_t sa = sbase + (uint32_t)(s * Cfg::STAGE_BYTES), sb = sa + Cfg::A_BYTES;
                const int k = kt * TC_K;
#pragma unroll
                for (int q = tid; q < TC_M * 8; q += TC_PRODUCERS) {
                    const int r = q >> 3, c = q & 7;
                    const uint32_t off = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
                    cp_async16_zfill(sa + off, la.src(m0 + r, k + c * 8, Kred), base);
                    if (r < BN) cp_async16_zfill(sb + off, lb.src(n0 + r, k + c * 8, Kred), base);
                }
            }
            cp_async_commit_group();
            if (kt >= TC_LAG) signal(kt - TC_LAG);
        }
        cp_async_wait_group<0>();
        // ---- epilogue: wait for the last commit, read the accumulators (a
        // warp-uniform decision: tcgen05.ld is a whole-warp instruction)
        bool bad = s_fail;
        if (!bad && !gsvr::mbar_wait_bounded(&done, 0u, kTcWaitNs)) bad = true;
        bad = __any_sync(0xffffffffu, bad);
        if (bad) s_fail = 1;
        tc_fence_after();
        if (!bad) {
            const int row = m0 + warp * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float f[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) f[t] = __uint_as_float(v[t]);
                ep.vec32(row, n0 + c0, f);
            }
        }
    } else if (lane == 0) {
        // ---- MMA issuer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % S;
            if (s_fail || !gsvr::mbar_wait_bounded(&full[s], (kt / S) & 1u, kTcWaitNs)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = sbase + (uint32_t)(s * Cfg::STAGE_BYTES), b0 = a0 + Cfg::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk)
                tc_mma(tmem, tc_smem_desc(a0 + kk * 32), tc_smem_desc(b0 + kk * 32), Cfg::IDESC,
                       (kt > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
        }
        tc_commit(&done);  // arrives once every MMA issued above has completed
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_fail) atomicOr(status, 4u);
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
}

// ---------------------------------------------- tcgen05 GEMM, TMA operands
// Same tile, swizzled layout, tensor-memory accumulation and epilogue as
// k_gemm_tc, with both operand tiles of a K step fetched by two tensor-map
// copies (cp.async.bulk.tensor) issued by one thread and counted on the
// stage's `full` barrier (expect_tx), so no thread waits on its own loads.
// Warp 0 (one lane) produces, warp 1 (one lane) issues the MMAs, warp 2 owns
// the tensor memory; all four warps run the epilogue.  Operand A is one of:
//   TMA_ROWS   a row-major [rows][K] matrix: box {64, 128} at (k, m0)
//   TMA_CONV   the forward im2col of a 3x3 / stride-2 / pad-1 convolution,
//              read from x [B][H][W][C] through a 4-D map that steps 2 input
//              pixels per output pixel: for K step k (tap t = k / C, channels
//              c0 = k % C) the box starts at (c0, kw - 1, 2 oh0 + kh - 1, b0);
//              negative and past-the-end coordinates read 0 (the padding)
//   TMA_GY2X2  the sub-pixel input-gradient operand, gy [B][OH][OW][C] through
//              a 4-D map: for K step k (d = k / C) the box starts at
//              (c0, d % 2, oh0 + d / 2, b0), past-the-end rows read 0
// For the 4-D kinds a 128-row tile is whole output rows of one image (P =
// OH OW >= 128) or whole images (P < 128), so that the box lands in shared
// memory in row order m = (b, oh, ow).
enum TmaKind { TMA_ROWS = 0, TMA_CONV = 1, TMA_GY2X2 = 2 };
struct TmaA {
    int kind;
    int lC;        // log2 channels per tap (4-D kinds)
    int lP, lOW;   // log2 of positions per image and of the output width (4-D kinds)
};
constexpr int TMA_THREADS = 128;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(gsvr::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(gsvr::smem_u32(bar))
        : "memory");
}

// Operand A outside the tensor (padding past the last tap): a batch index no
// tensor reaches, so the whole box reads 0.
constexpr int kTmaNowhere = 1 << 20;

template <class EP, int BN, int SW>
__global__ void __launch_bounds__(TMA_THREADS) k_gemm_tma(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, TmaA ta, EP ep,
                                                          int Kred, unsigned *status) {
    using Cfg = TcCfg<BN>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * BN;
    const uint32_t sbase = (gsvr::smem_u32(tc_raw) + 1023u) & ~1023u;
    const int nk = (Kred + TC_K - 1) / TC_K;
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gsvr::smem_u32(&s_tmem)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            gsvr::mbar_init(&full[i], 1);
            gsvr::mbar_init(&empty[i], 1);
        }
        gsvr::mbar_init(&done, 1);
        gsvr::fence_mbar_init();
        s_fail = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (warp == 0 && lane == 0) {
        // ---- producer
        int b0 = 0, oh0 = 0;
        if (ta.kind != TMA_ROWS) {
            b0 = m0 >> ta.lP;
            oh0 = (m0 - (b0 << ta.lP)) >> ta.lOW;
        }
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % S;
            if (kt >= S && !gsvr::mbar_wait_bounded(&empty[s], ((kt / S) - 1) & 1u, kTcWaitNs)) s_fail = 1;
            if (s_fail) break;
            const uint32_t sa = sbase + (uint32_t)(s * Cfg::STAGE_BYTES), sb = sa + Cfg::A_BYTES;
            gsvr::mbar_arrive_expect_tx(&full[s], (uint32_t)Cfg::STAGE_BYTES);
            // SW = 128: one box of 64 K per operand; SW = 64: two boxes of 32 K
            // (each a 64-byte-swizzled block of its own: A 8 KB, B BN x 64 B)
#pragma unroll
            for (int h = 0; h < 128 / SW; ++h) {
                const int k = kt * TC_K + h * (SW / 2);
                const uint32_t da = sa + (uint32_t)(h * TC_M * SW), db = sb + (uint32_t)(h * BN * SW);
                if (ta.kind == TMA_ROWS) {
                    tma_load_2d(da, &mapA, k, m0, &full[s]);
                } else {
                    const int t = k >> ta.lC, c0 = k & ((1 << ta.lC) - 1);
                    if (ta.kind == TMA_CONV) {
                        const int kh = (t * 11) >> 5, kw = t - 3 * kh;  // t / 3 for t < 9
                        tma_load_4d(da, &mapA, c0, kw - 1, 2 * oh0 + kh - 1, t < 9 ? b0 : kTmaNowhere, &full[s]);
                    } else {
                        tma_load_4d(da, &mapA, c0, t & 1, oh0 + (t >> 1), t < 4 ? b0 : kTmaNowhere, &full[s]);
                    }
                }
                tma_load_2d(db, &mapB, k, n0, &full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % S;
            if (s_fail || !gsvr::mbar_wait_bounded(&full[s], (kt / S) & 1u, kTcWaitNs)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = sbase + (uint32_t)(s * Cfg::STAGE_BYTES), b0 = a0 + Cfg::A_BYTES;
            if (SW == 128) {
#pragma unroll
                for (int kk = 0; kk < TC_K / 16; ++kk)
                    tc_mma(tmem, tc_smem_desc(a0 + kk * 32), tc_smem_desc(b0 + kk * 32), Cfg::IDESC,
                           (kt > 0 || kk > 0) ? 1u : 0u);
            } else {
#pragma unroll
                for (int kk = 0; kk < TC_K / 16; ++kk) {
                    const uint32_t h = kk >> 1, o = (kk & 1) * 32;
                    tc_mma(tmem, tc_smem_desc64(a0 + h * TC_M * 64 + o), tc_smem_desc64(b0 + h * BN * 64 + o),
                           Cfg::IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
                }
            }
            tc_commit(&empty[s]);
        }
        tc_commit(&done);  // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // ---- epilogue (all four warps; the decision is warp-uniform)
    bool bad = s_fail;
    if (!bad && !gsvr::mbar_wait_bounded(&done, 0u, kTcWaitNs)) bad = true;
    bad = __any_sync(0xffffffffu, bad);
    if (bad) s_fail = 1;
    tc_fence_after();
    if (!bad) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float f[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) f[t] = __uint_as_float(v[t]);
            ep.vec32(row, n0 + c0, f);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_fail) atomicOr(status, 4u);
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
}

// Host: the CUDA driver API's tensor-map encoder, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}
// bfloat16 tensor map with the 128-byte swizzle; dims / strides innermost
// first (strides in bytes, rank - 1 of them), zero fill outside the tensor.
bool encode_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides,
                const uint32_t *box, const uint32_t *estride, int sw = 128) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base),
               reinterpret_cast<const cuuint64_t *>(dims), reinterpret_cast<const cuuint64_t *>(strides),
               reinterpret_cast<const cuuint32_t *>(box), reinterpret_cast<const cuuint32_t *>(estride),
               CU_TENSOR_MAP_INTERLEAVE_NONE, sw == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
// [rows][K] row-major bfloat16 (K % 8 == 0, 16-byte aligned), box {sw / 2, box_rows}
bool map_rows(CUtensorMap *m, const bf16 *p, int rows, int K, int box_rows, int sw = 128) {
    const uint64_t dims[2] = {(uint64_t)K, (uint64_t)rows}, strides[1] = {(uint64_t)K * 2};
    const uint32_t box[2] = {(uint32_t)(sw / 2), (uint32_t)box_rows}, es[2] = {1, 1};
    return encode_map(m, p, 2, dims, strides, box, es, sw);
}
int ilog2_exact(int v) {  // log2 of a power of two, else -1
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
// Tile of `rows` (a power of two) output positions as (images bb) x (rows
// bh) x (all OW columns); false when the output grid does not split that way.
bool tile_rows(const ConvShape &s, int &bh, int &bb, int rows = TC_M) {
    const int P = s.OH * s.OW;
    if (ilog2_exact(s.OW) < 0 || ilog2_exact(P) < 0 || s.OW > rows) return false;
    if (P >= rows) {
        bh = rows / s.OW;
        bb = 1;
    } else {
        bh = s.OH;
        bb = rows / P;
    }
    return true;
}

template <class EP, int BN, int SW>
cudaError_t launch_tma_n(const CUtensorMap &mA, const CUtensorMap &mB, TmaA ta, EP ep, int rows, int cols, int Kred,
                         unsigned *status, cudaStream_t st) {
    const dim3 grid((rows + TC_M - 1) / TC_M, (cols + BN - 1) / BN);
    cudaError_t e =
        cudaFuncSetAttribute(k_gemm_tma<EP, BN, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN>::SMEM);
    if (e) return e;
    k_gemm_tma<EP, BN, SW><<<grid, TMA_THREADS, TcCfg<BN>::SMEM, st>>>(mA, mB, ta, ep, Kred, status);
    return cudaGetLastError();
}
// sw: the swizzle span of both maps (128: boxes of 64 K, 64: boxes of 32 K)
template <class EP>
cudaError_t launch_tma(const CUtensorMap &mA, const CUtensorMap &mB, TmaA ta, EP ep, int rows, int cols, int Kred,
                       unsigned *status, cudaStream_t st, int sw = 128) {
    if (cols <= 64)
        return sw == 64 ? launch_tma_n<EP, 64, 64>(mA, mB, ta, ep, rows, cols, Kred, status, st)
                        : launch_tma_n<EP, 64, 128>(mA, mB, ta, ep, rows, cols, Kred, status, st);
    return sw == 64 ? launch_tma_n<EP, 128, 64>(mA, mB, ta, ep, rows, cols, Kred, status, st)
                    : launch_tma_n<EP, 128, 128>(mA, mB, ta, ep, rows, cols, Kred, status, st);
}

// ------------------------------------ tcgen05 weight gradient (MN-major)
// dW[co][n] += sum over positions m of gy[m][co] X[m][n], n = (tap, ci) the
// im2col column: the reduction runs over positions, which are the outer index
// of both operands in memory, so both tiles are MN-major: per 64-position K
// step, gy [M][Co] gives two tensor-map boxes of 64 channels x 64 positions
// (channels contiguous, 128-byte swizzle) and the input x gives BN / 64 boxes
// of 64 input channels x 64 positions of one tap (the stride-2 4-D map of the
// forward, its 64-position step whole output rows or images).  The smem
// descriptors of the MN-major 128-byte-swizzled layout take the stride between
// 64-element channel atoms (8 KB here) as leading byte offset and the stride
// between 8-position groups (1024 B) as stride byte offset; the instruction
// descriptor sets transpose A and B.  The position range is split over
// blockIdx.z; each split adds its tile into dw with float4 atomics.
constexpr int WG_K = 64;  // positions per K step
__device__ __forceinline__ uint64_t tc_smem_desc_mn(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(8192u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}
// MN-major, 64-byte swizzle: 32-element atoms 4 KB apart (leading), 8-position
// groups 512 B apart (stride)
__device__ __forceinline__ uint64_t tc_smem_desc_mn64(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(4096u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)4u << 61);
}
// XSW: swizzle span of the input's boxes (128: 64 channels of a tap per box,
// 64: 32 channels, for Ci = 32)
template <int BN, int XSW>
__global__ void __launch_bounds__(TMA_THREADS) k_wgrad_tma(const __grid_constant__ CUtensorMap mapG,
                                                           const __grid_constant__ CUtensorMap mapX, TmaA tx,
                                                           float *__restrict__ dw, int Co, int K9, int nk_total,
                                                           int steps, unsigned *status) {
    using Cfg = TcCfg<BN>;
    constexpr int S = Cfg::STAGES;
    constexpr uint32_t IDESC = Cfg::IDESC | (1u << 15) | (1u << 16);  // A and B MN-major
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int co0 = blockIdx.x * TC_M, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * steps, ke = min(nk_total, kb + steps), nk = ke - kb;
    const uint32_t sbase = (gsvr::smem_u32(tc_raw) + 1023u) & ~1023u;
    if (nk <= 0) return;
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gsvr::smem_u32(&s_tmem)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            gsvr::mbar_init(&full[i], 1);
            gsvr::mbar_init(&empty[i], 1);
        }
        gsvr::mbar_init(&done, 1);
        gsvr::fence_mbar_init();
        s_fail = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapG)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapX)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (warp == 0 && lane == 0) {
        for (int i = 0; i < nk; ++i) {
            const int s = i % S;
            if (i >= S && !gsvr::mbar_wait_bounded(&empty[s], ((i / S) - 1) & 1u, kTcWaitNs)) s_fail = 1;
            if (s_fail) break;
            const uint32_t sa = sbase + (uint32_t)(s * Cfg::STAGE_BYTES), sb = sa + Cfg::A_BYTES;
            const int m = (kb + i) * WG_K;
            const int b0 = m >> tx.lP, oh0 = (m - (b0 << tx.lP)) >> tx.lOW;
            gsvr::mbar_arrive_expect_tx(&full[s], (uint32_t)Cfg::STAGE_BYTES);
            tma_load_2d(sa, &mapG, co0, m, &full[s]);
            tma_load_2d(sa + 8192u, &mapG, co0 + 64, m, &full[s]);
#pragma unroll
            for (int a = 0; a < BN / (XSW / 2); ++a) {
                const int n = n0 + (XSW / 2) * a, t = n >> tx.lC, c0 = n & ((1 << tx.lC) - 1);
                const int kh = (t * 11) >> 5, kw = t - 3 * kh;
                tma_load_4d(sb + (uint32_t)(a * (XSW / 2) * WG_K * 2), &mapX, c0, kw - 1, 2 * oh0 + kh - 1,
                            t < 9 ? b0 : kTmaNowhere, &full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        for (int i = 0; i < nk; ++i) {
            const int s = i % S;
            if (s_fail || !gsvr::mbar_wait_bounded(&full[s], (i / S) & 1u, kTcWaitNs)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = sbase + (uint32_t)(s * Cfg::STAGE_BYTES), b0 = a0 + Cfg::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < WG_K / 16; ++kk)  // 16 positions = two 8-position groups
                tc_mma(tmem, tc_smem_desc_mn(a0 + kk * 2048),
                       XSW == 128 ? tc_smem_desc_mn(b0 + kk * 2048) : tc_smem_desc_mn64(b0 + kk * 1024), IDESC,
                       (i > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
        }
        tc_commit(&done);
    }
    __syncwarp();
    bool bad = s_fail;
    if (!bad && !gsvr::mbar_wait_bounded(&done, 0u, kTcWaitNs)) bad = true;
    bad = __any_sync(0xffffffffu, bad);
    if (bad) s_fail = 1;
    tc_fence_after();
    if (!bad) {
        const int co = co0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN && n0 + c0 < K9; c0 += 32) {  // K9 % 32 == 0
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (co < Co) {
                float4 *d = reinterpret_cast<float4 *>(dw + (size_t)co * K9 + n0 + c0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    atomicAdd(d + j, make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3])));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_fail) atomicOr(status, 4u);
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
}

// db[c] += sum over rows m of g[m][c] (bfloat16 [M][C], C % 8 == 0): block
// (x, y) covers channels 256 y .. 256 y + 255 (lane l: 8 channels by one
// 16-byte load) over the rows m = x, x + gridDim.x * 8, ... of its 8 warps
// (warp w from row x * 8 + w); the warps' sums meet in shared memory, one
// atomic per (block, channel).
// lpr lanes per row (a power of two: C / 8 when that is one below 32, else
// 32 with the lanes past the channels idle), 32 / lpr rows per warp step.
__global__ void __launch_bounds__(256) k_colsum_bf16_add(const bf16 *__restrict__ g, int M, int C, int lpr,
                                                         float *__restrict__ db) {
    __shared__ float red[8][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, rpw = 32 / lpr;
    const int cg = lane % lpr, sub = lane / lpr, c0 = blockIdx.y * 256 + cg * 8;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (c0 < C) {
        for (int m = (blockIdx.x * 8 + warp) * rpw + sub; m < M; m += gridDim.x * 8 * rpw) {
            const uint4 u = *reinterpret_cast<const uint4 *>(g + (size_t)m * C + c0);
            const bf16 *h = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] += __bfloat162float(h[e]);
        }
    }
    for (int off = lpr; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] += __shfl_xor_sync(0xffffffffu, v[e], off);
    if (lane < lpr) {
#pragma unroll
        for (int e = 0; e < 8; ++e) red[warp][lane * 8 + e] = v[e];
    }
    __syncthreads();
    const int c = blockIdx.y * 256 + threadIdx.x;
    if (threadIdx.x < lpr * 8 && c < C) {
        float t = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) t += red[w8][threadIdx.x];
        atomicAdd(&db[c], t);
    }
}

// Latched status of the tcgen05 kernels that the layer primitives launch
// (bit 4: a bounded wait ran out); gsvr_cnn_sync_status(NULL) reads and clears it.
__device__ unsigned g_tc_status;
unsigned *tc_status_word() {
    static unsigned *p = nullptr;
    if (!p) cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_tc_status);
    return p;
}
// The tensor-memory path serves GEMMs whose output has at least this many
// columns (narrower outputs waste most of the 128-column tile).
constexpr int kTcMinCols = 64;

template <class LA, class LB, class EP, int BN>
cudaError_t gemm_tc_n(LA la, LB lb, EP ep, int rows, int cols, int Kred, const void *base, unsigned *status,
                      cudaStream_t st) {
    const dim3 grid((rows + TC_M - 1) / TC_M, (cols + BN - 1) / BN);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<LA, LB, EP, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcCfg<BN>::SMEM);
    if (e) return e;
    k_gemm_tc<LA, LB, EP, BN><<<grid, TC_THREADS, TcCfg<BN>::SMEM, st>>>(la, lb, ep, Kred, base, status);
    return cudaGetLastError();
}
// base: any valid global address (stands in for the zero-filled copies)
template <class LA, class LB, class EP>
cudaError_t gemm_tc(LA la, LB lb, EP ep, int rows, int cols, int Kred, const void *base, unsigned *status,
                    cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || Kred <= 0) return cudaSuccess;
    return cols <= 64 ? gemm_tc_n<LA, LB, EP, 64>(la, lb, ep, rows, cols, Kred, base, status, st)
                      : gemm_tc_n<LA, LB, EP, 128>(la, lb, ep, rows, cols, Kred, base, status, st);
}

// Dense C[m][n] (float32, row-major, ld = N) epilogue for the standalone GEMM.
struct EpiDense {
    float *c;
    int M, N;
    __device__ void operator()(int m, int n, float v) const {
        if (m < M && n < N) c[(size_t)m * N + n] = v;
    }
    __device__ void vec8(int m, int n0, const float *v) const {
        if (m >= M) return;
        if (n0 + 8 > N || (N & 3)) {
            for (int j = 0; j < 8; ++j) (*this)(m, n0 + j, v[j]);
            return;
        }
        float4 *d = reinterpret_cast<float4 *>(c + (size_t)m * N + n0);
        d[0] = make_float4(v[0], v[1], v[2], v[3]);
        d[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    __device__ void vec32(int m, int n0, const float *v) const {
#pragma unroll
        for (int j = 0; j < 32; j += 8) vec8(m, n0 + j, v + j);
    }
};

// ------------------------------------------- reduction-major operands (wgrad)
// Loaders of the transposed form: 8 bfloat16 values (kr, c0 .. c0 + 7) of an
// operand whose reduction index kr is the slow one; zero for kr >= kr_end.
struct LoadRowsT {  // p[kr][ld], columns c < cols (cols % 8 == 0)
    const bf16 *p;
    int ld, cols;
    __device__ uint4 operator()(int kr, int c0, int kr_end) const {
        if (kr >= kr_end || c0 >= cols) return zero4();
        return *reinterpret_cast<const uint4 *>(p + (size_t)kr * ld + c0);
    }
};
struct LoadIm2colRowT {  // X(m = kr, k = c0 ..), the bias column K reads 1
    LoadIm2col x;
    int K;
    __device__ uint4 operator()(int kr, int c0, int kr_end) const {
        if (kr >= kr_end || c0 > K) return zero4();
        if (c0 == K) return make_uint4(0x3F80u, 0u, 0u, 0u);  // bfloat16 1.0, then zeros
        return x(kr, c0, K);
    }
};

__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

constexpr int LDA_T = BM + 8, LDB_T = BN + 8;  // reduction-major tiles, padded rows

// C[rows][cols] = sum over the reduction range of A(row, k) B(col, k), with both
// operands loaded reduction-major (coalesced along rows / cols) into shared
// memory and read with ldmatrix.trans.
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(GT) k_gemm_t(LA la, LB lb, EP ep, int Kred, int ksplit) {
    __shared__ __align__(16) bf16 sA[2][BK * LDA_T];
    __shared__ __align__(16) bf16 sB[2][BK * LDB_T];
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
    // A tile: 32 k x 128 rows = 512 chunks of 8 (two per thread); B: 32 x 64 = 256 (one)
    auto load = [&](int k) {
        ra0 = la(k + (tid >> 4), m0 + (tid & 15) * 8, ke);
        ra1 = la(k + 16 + (tid >> 4), m0 + (tid & 15) * 8, ke);
        rb0 = lb(k + (tid >> 3), n0 + (tid & 7) * 8, ke);
    };
    auto store = [&](int buf) {
        *reinterpret_cast<uint4 *>(&sA[buf][(tid >> 4) * LDA_T + (tid & 15) * 8]) = ra0;
        *reinterpret_cast<uint4 *>(&sA[buf][(16 + (tid >> 4)) * LDA_T + (tid & 15) * 8]) = ra1;
        *reinterpret_cast<uint4 *>(&sB[buf][(tid >> 3) * LDB_T + (tid & 7) * 8]) = rb0;
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
            const int q = lane >> 3, l7 = lane & 7;
#pragma unroll
            for (int i = 0; i < 2; ++i)
                ldsm_x4_t(a[i], &sA[buf][(kk + (q >> 1) * 8 + l7) * LDA_T + wm * 32 + i * 16 + (q & 1) * 8]);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t t[4];
                ldsm_x4_t(t, &sB[buf][(kk + (q & 1) * 8 + l7) * LDB_T + wn * 32 + j * 16 + (q >> 1) * 8]);
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
cudaError_t gemm_t(LA la, LB lb, EP ep, int rows, int cols, int Kred, int ksplit, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || Kred <= 0) return cudaSuccess;
    ksplit = std::max(BK, (ksplit + BK - 1) / BK * BK);
    const dim3 grid((rows + BM - 1) / BM, (cols + BN - 1) / BN, (Kred + ksplit - 1) / ksplit);
    if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidValue;
    k_gemm_t<LA, LB, EP><<<grid, GT, 0, st>>>(la, lb, ep, Kred, ksplit);
    return cudaGetLastError();
}

// ------------------------------------------- input gradient, sub-pixel form
// Output position (i, j) feeds the 2 x 2 input pixels (2i + ph, 2j + pw): for
// ih = 2i the tap is kh = 1 from oh = i; for ih = 2i + 1 the taps are kh = 2
// from oh = i and kh = 0 from oh = i + 1 (likewise along w).  So one GEMM per
// layer: rows m = (b, i, j), reduction k = (dy, dx, co) over gy[b][i + dy][j + dx],
// columns n = (ph, pw, ci), with the sub-pixel weights
//   W'[(ph, pw, ci)][(dy, dx, co)] = W[co][kh(ph, dy)][kw(pw, dx)][ci]
// (zero where (ph, dy) has no tap: 9 of the 16 blocks are nonzero).
__device__ __forceinline__ int subpixel_tap(int p, int d) { return p == 0 ? (d == 0 ? 1 : -1) : (d == 0 ? 2 : 0); }
struct LoadGy2x2 {  // A(m, k = (dy, dx, co)) = gy[b][i + dy][j + dx][co .. co + 7]
    const bf16 *gy;
    ConvShape s;
    int rows;
    __device__ uint4 operator()(int m, int k0, int k_end) const {
        if (m >= rows || k0 >= k_end) return zero4();
        int d, co, b, i, j;
        chan_split(k0, s.Co, s.lCo, d, co);
        pos_split(s, m, b, i, j);
        const int oh = i + (d >> 1), ow = j + (d & 1);
        if (oh >= s.OH || ow >= s.OW) return zero4();
        return *reinterpret_cast<const uint4 *>(gy + (((size_t)b * s.OH + oh) * s.OW + ow) * s.Co + co);
    }
    __device__ const bf16 *src(int m, int k0, int k_end) const {
        if (m >= rows || k0 >= k_end) return nullptr;
        int d, co, b, i, j;
        chan_split(k0, s.Co, s.lCo, d, co);
        pos_split(s, m, b, i, j);
        const int oh = i + (d >> 1), ow = j + (d & 1);
        if (oh >= s.OH || ow >= s.OW) return nullptr;
        return gy + (((size_t)b * s.OH + oh) * s.OW + ow) * s.Co + co;
    }
};
// W' [4 Ci][4 Co] from W [Co][3][3][Ci]
__global__ void k_subpixel_weights(const bf16 *__restrict__ w, int Ci, int Co, bf16 *__restrict__ wp) {
    const int64_t n = (int64_t)16 * Ci * Co;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % (4 * Co)), r = (int)(e / (4 * Co));
        const int d = k / Co, co = k - d * Co, ph_pw = r / Ci, ci = r - ph_pw * Ci;
        const int kh = subpixel_tap(ph_pw >> 1, d >> 1), kw = subpixel_tap(ph_pw & 1, d & 1);
        wp[e] = (kh < 0 || kw < 0) ? __float2bfloat16(0.f) : w[(((size_t)co * 3 + kh) * 3 + kw) * Ci + ci];
    }
}
struct EpiDx2x2 {  // dx[b][2i + ph][2j + pw][ci] = acc (times mask > 0), inside the input only
    bf16 *dx;
    float *dx32;
    const bf16 *mask;
    ConvShape s;
    int rows;
    __device__ void operator()(int m, int n, float v) const {
        if (m >= rows || n >= 4 * s.Ci) return;
        int q, ci, b, i, j;
        chan_split(n, s.Ci, s.lCi, q, ci);
        pos_split(s, m, b, i, j);
        const int ih = 2 * i + (q >> 1), iw = 2 * j + (q & 1);
        if (ih >= s.H || iw >= s.W) return;
        const size_t e = (((size_t)b * s.H + ih) * s.W + iw) * s.Ci + ci;
        if (mask && !(__bfloat162float(mask[e]) > 0.f)) v = 0.f;
        dx[e] = __float2bfloat16(v);
        if (dx32) dx32[e] = v;
    }
    // columns n0 .. n0 + 31 as four 8-column groups: every mask load is
    // issued before any store
    __device__ void vec32(int m, int n0, const float *v) const {
        if (m >= rows) return;
        int b, i, j;
        pos_split(s, m, b, i, j);
        size_t e[4];
        bool ok[4];
        uint4 mk[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            int q, ci;
            chan_split(n0 + 8 * g, s.Ci, s.lCi, q, ci);
            const int ih = 2 * i + (q >> 1), iw = 2 * j + (q & 1);
            ok[g] = n0 + 8 * g < 4 * s.Ci && ih < s.H && iw < s.W;
            e[g] = ok[g] ? (((size_t)b * s.H + ih) * s.W + iw) * s.Ci + ci : 0;
            mk[g] = (ok[g] && mask) ? __ldg(reinterpret_cast<const uint4 *>(mask + e[g])) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            if (!ok[g]) continue;
            const bf16 *mb = reinterpret_cast<const bf16 *>(&mk[g]);
            float o[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) o[t] = (mask && !(__bfloat162float(mb[t]) > 0.f)) ? 0.f : v[8 * g + t];
            *reinterpret_cast<uint4 *>(dx + e[g]) = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]),
                                                               pack_bf16x2(o[4], o[5]), pack_bf16x2(o[6], o[7]));
            if (dx32) {
                reinterpret_cast<float4 *>(dx32 + e[g])[0] = make_float4(o[0], o[1], o[2], o[3]);
                reinterpret_cast<float4 *>(dx32 + e[g])[1] = make_float4(o[4], o[5], o[6], o[7]);
            }
        }
    }
};

// ------------------------------------------------------- element kernels
__global__ void k_to_bf16(const float *__restrict__ a, int64_t n, bf16 *__restrict__ b) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = __float2bfloat16(a[e]);
}

// First layer (one input channel, 32 outputs).  Forward: a thread per output
// position gathers its 3 x 3 patch once and computes all 32 channels, the
// weights read from shared memory as float4 that every lane of the warp
// shares (broadcast); the 64 output bytes of a position are four 16-byte
// stores.  The weight gradient (below) uses four threads per position.
__device__ __forceinline__ void conv1_patch(const bf16 *__restrict__ x, const ConvShape &s, int m, float xv[9]) {
    int b, oh, ow;
    pos_split(s, m, b, oh, ow);
#pragma unroll
    for (int kh = 0; kh < 3; ++kh)
#pragma unroll
        for (int kw = 0; kw < 3; ++kw) {
            const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
            xv[kh * 3 + kw] = (ih >= 0 && ih < s.H && iw >= 0 && iw < s.W)
                                  ? __bfloat162float(x[((size_t)b * s.H + ih) * s.W + iw])
                                  : 0.f;
        }
}
// shared-memory float4 read kept inside its loop (a volatile asm is not
// hoisted), so that loop-invariant weights are re-read instead of held in
// registers
__device__ __forceinline__ float4 lds_f4(const float4 *p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_addr(p)));
    return v;
}
__global__ void __launch_bounds__(256) k_conv1_fwd(const bf16 *__restrict__ x, ConvShape s,
                                                   const bf16 *__restrict__ w, const float *__restrict__ bias,
                                                   bf16 *__restrict__ y) {
    __shared__ float4 ws4[32 * 9 / 4];  // [co][tap] row-major: channel pair (2c, 2c + 1) = floats 18 c .. 18 c + 17
    __shared__ float bs[32];
    float *ws = reinterpret_cast<float *>(ws4);
    for (int e = threadIdx.x; e < 32 * 9; e += blockDim.x) ws[e] = __bfloat162float(w[e]);
    for (int e = threadIdx.x; e < 32; e += blockDim.x) bs[e] = bias[e];
    __syncthreads();
    const int64_t M = (int64_t)s.B * s.OH * s.OW;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        float xv[9];
        conv1_patch(x, s, (int)m, xv);
        uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)m * 32);
#pragma unroll
        for (int g = 0; g < 4; ++g) {  // channels 8 g .. 8 g + 7: floats 72 g .. 72 g + 71 = 18 float4
            float wv[72];
#pragma unroll
            for (int i = 0; i < 18; ++i) {
                const float4 t = lds_f4(&ws4[18 * g + i]);
                wv[4 * i] = t.x;
                wv[4 * i + 1] = t.y;
                wv[4 * i + 2] = t.z;
                wv[4 * i + 3] = t.w;
            }
            uint32_t pk[4];
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
                float v0 = bs[8 * g + c], v1 = bs[8 * g + c + 1];
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    v0 = fmaf(wv[c * 9 + k], xv[k], v0);
                    v1 = fmaf(wv[(c + 1) * 9 + k], xv[k], v1);
                }
                pk[c / 2] = pack_bf16x2(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
            }
            dst[g] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
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
// C[m][n] = sum_k A(m, k) B(n, k) in float32 with A(m, k) = A[m sam + k sak],
// B(n, k) = B[n sbn + k sbk]: 64 x 64 tiles through shared memory (loads
// coalesced along whichever index has unit stride), 4 x 4 outputs per thread.
template <class EP>
__global__ void __launch_bounds__(256) k_sgemm(const float *__restrict__ A, int sam, int sak,
                                               const float *__restrict__ Bm, int sbn, int sbk, int M, int N, int Kfull,
                                               int ksplit, EP ep) {
    __shared__ __align__(16) float As[2][16][68];
    __shared__ __align__(16) float Bs[2][16][68];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int kbeg = blockIdx.z * ksplit, K = min(Kfull, kbeg + ksplit);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float ra[4], rb[4];
    // element q of this thread's share: unit-stride index fastest across threads
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int mm = sak == 1 ? (e >> 4) : (e & 63), kk = sak == 1 ? (e & 15) : (e >> 6);
            const int m = m0 + mm, k = k0 + kk;
            ra[q] = (m < M && k < K) ? A[(size_t)m * sam + (size_t)k * sak] : 0.f;
            const int nn = sbk == 1 ? (e >> 4) : (e & 63), kb = sbk == 1 ? (e & 15) : (e >> 6);
            const int n = n0 + nn, k2 = k0 + kb;
            rb[q] = (n < N && k2 < K) ? Bm[(size_t)n * sbn + (size_t)k2 * sbk] : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int mm = sak == 1 ? (e >> 4) : (e & 63), kk = sak == 1 ? (e & 15) : (e >> 6);
            As[buf][kk][mm] = ra[q];
            const int nn = sbk == 1 ? (e >> 4) : (e & 63), kb = sbk == 1 ? (e & 15) : (e >> 6);
            Bs[buf][kb][nn] = rb[q];
        }
    };
    if (kbeg < K) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < K; k0 += 16) {
        const bool more = k0 + 16 < K;
        if (more) load(k0 + 16);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ep(m0 + ty * 4 + i, n0 + tx * 4 + j, acc[i][j]);
}
struct EpiFc {  // out = relu?(acc + bias[n]), z (may be null) keeps the pre-activation
    float *out, *z;
    const float *bias;
    int M, N, relu;
    __device__ void operator()(int m, int n, float v) const {
        if (m >= M || n >= N) return;
        v += bias[n];
        if (z) z[(size_t)m * N + n] = v;
        out[(size_t)m * N + n] = relu ? fmaxf(v, 0.f) : v;
    }
};
struct EpiF {  // out[m][n] = acc, times (zin > 0) when zin is given
    float *out;
    const float *zin;
    int M, N;
    __device__ void operator()(int m, int n, float v) const {
        if (m >= M || n >= N) return;
        if (zin && !(zin[(size_t)m * N + n] > 0.f)) v = 0.f;
        out[(size_t)m * N + n] = v;
    }
};
struct EpiPart {  // part[split][m][n] = acc (split = blockIdx.z)
    float *part;
    int M, N;
    __device__ void operator()(int m, int n, float v) const {
        if (m < M && n < N) part[((size_t)blockIdx.z * M + m) * N + n] = v;
    }
};
template <class EP>
void sgemm(const float *A, int sam, int sak, const float *B, int sbn, int sbk, int M, int N, int K, EP ep,
           cudaStream_t st, int splits = 1) {
    const int ks = (K + splits - 1) / splits;
    k_sgemm<EP><<<dim3((M + 63) / 64, (N + 63) / 64, splits), 256, 0, st>>>(A, sam, sak, B, sbn, sbk, M, N, K, ks,
                                                                           ep);
}
// out = relu?(sum over splits of part + bias), z keeps the pre-activation
__global__ void k_fc_finish(const float *__restrict__ part, int splits, int M, int N, const float *__restrict__ bias,
                            int relu, float *__restrict__ z, float *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x) {
        float v = bias[e % N];
        for (int q = 0; q < splits; ++q) v += part[(size_t)q * M * N + e];
        if (z) z[e] = v;
        out[e] = relu ? fmaxf(v, 0.f) : v;
    }
}
constexpr int kFc1Splits = 8;
// out[e] = sum over splits of part[split][e]
__global__ void k_part_sum(const float *__restrict__ part, int splits, int64_t n, float *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int q = 0; q < splits; ++q) v += part[(size_t)q * n + e];
        out[e] = v;
    }
}
// db[j] += sum_b d[b][j]: block (x, y) takes columns 32 x .. 32 x + 31 (a
// lane each) and rows 32 y .. 32 y + 31 (4 per warp); the warps meet in
// shared memory, one atomic per (block, column).
__global__ void __launch_bounds__(256) k_colsum_add(const float *__restrict__ d, int B, int J,
                                                    float *__restrict__ db) {
    __shared__ float red[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, j = blockIdx.x * 32 + lane;
    float v = 0.f;
    if (j < J) {
        const int b1 = min(B, (int)blockIdx.y * 32 + 32);
        for (int b = blockIdx.y * 32 + warp; b < b1; b += 8) v += d[(size_t)b * J + j];
    }
    red[warp][lane] = v;
    __syncthreads();
    if (warp == 0 && j < J) {
        float t = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) t += red[w8][lane];
        atomicAdd(&db[j], t);
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

int log2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return (1 << l) == v ? l : -1;
}
ConvShape conv_shape(int B, int H, int W, int Ci, int Co) {
    const int OH = (H + 1) / 2, OW = (W + 1) / 2;
    return ConvShape{B, H, W, Ci, OH, OW, Co, log2_exact(OW), log2_exact(OH), log2_exact(Ci), log2_exact(Co)};
}

// --------------------------------------------------------- conv operations
cudaError_t conv_forward(const bf16 *x, const ConvShape &s, const bf16 *w, const float *bias, int relu, bf16 *y,
                         float *y32, unsigned *status, cudaStream_t st) {
    const int M = s.B * s.OH * s.OW, K = 9 * s.Ci;
    if (s.Ci == 1 && s.Co == 32 && relu && !y32) {
        k_conv1_fwd<<<blocks_for(M, 256 * 2), 256, 0, st>>>(x, s, w, bias, y);
        return cudaGetLastError();
    }
    if (s.Co >= kTcMinCols) {
        const EpiConv ep{y, y32, bias, M, s.Co, relu};
        int bh, bb;
        const int sw = s.Ci % 64 == 0 ? 128 : s.Ci == 32 ? 64 : 0;  // box of sw / 2 channels
        if (sw && tile_rows(s, bh, bb)) {
            CUtensorMap mA, mB;
            const uint64_t dims[4] = {(uint64_t)s.Ci, (uint64_t)s.W, (uint64_t)s.H, (uint64_t)s.B};
            const uint64_t strides[3] = {(uint64_t)s.Ci * 2, (uint64_t)s.W * s.Ci * 2, (uint64_t)s.H * s.W * s.Ci * 2};
            const uint32_t box[4] = {(uint32_t)(sw / 2), (uint32_t)(2 * s.OW), (uint32_t)(2 * bh), (uint32_t)bb};
            const uint32_t es[4] = {1, 2, 2, 1};
            if (encode_map(&mA, x, 4, dims, strides, box, es, sw) &&
                map_rows(&mB, w, s.Co, K, s.Co <= 64 ? 64 : 128, sw))
                return launch_tma(mA, mB, TmaA{TMA_CONV, ilog2_exact(s.Ci), ilog2_exact(s.OH * s.OW), ilog2_exact(s.OW)},
                                  ep, M, s.Co, K, status, st, sw);
        }
        return gemm_tc(LoadIm2col{x, s, M, K}, LoadRows{w, s.Co, K}, ep, M, s.Co, K, w, status, st);
    }
    return gemm(LoadIm2col{x, s, M, K}, LoadRows{w, s.Co, K}, EpiConv{y, y32, bias, M, s.Co, relu}, M, s.Co, K, K,
                st);
}

cudaError_t conv_dgrad(const bf16 *gy, const ConvShape &s, const bf16 *w, bf16 *wp, const bf16 *mask, bf16 *dx,
                       float *dx32, unsigned *status, cudaStream_t st) {
    k_subpixel_weights<<<blocks_for((int64_t)16 * s.Ci * s.Co), 256, 0, st>>>(w, s.Ci, s.Co, wp);
    const int rows = s.B * s.OH * s.OW;
    if (4 * s.Ci >= kTcMinCols) {
        const EpiDx2x2 ep{dx, dx32, mask, s, rows};
        int bh, bb;
        if (s.Co % 64 == 0 && tile_rows(s, bh, bb)) {
            CUtensorMap mA, mB;
            const uint64_t dims[4] = {(uint64_t)s.Co, (uint64_t)s.OW, (uint64_t)s.OH, (uint64_t)s.B};
            const uint64_t strides[3] = {(uint64_t)s.Co * 2, (uint64_t)s.OW * s.Co * 2,
                                         (uint64_t)s.OH * s.OW * s.Co * 2};
            const uint32_t box[4] = {(uint32_t)TC_K, (uint32_t)s.OW, (uint32_t)bh, (uint32_t)bb};
            const uint32_t es[4] = {1, 1, 1, 1};
            if (encode_map(&mA, gy, 4, dims, strides, box, es) &&
                map_rows(&mB, wp, 4 * s.Ci, 4 * s.Co, 4 * s.Ci <= 64 ? 64 : 128))
                return launch_tma(mA, mB,
                                  TmaA{TMA_GY2X2, ilog2_exact(s.Co), ilog2_exact(s.OH * s.OW), ilog2_exact(s.OW)}, ep,
                                  rows, 4 * s.Ci, 4 * s.Co, status, st);
        }
        return gemm_tc(LoadGy2x2{gy, s, rows}, LoadRows{wp, 4 * s.Ci, 4 * s.Co}, ep, rows, 4 * s.Ci, 4 * s.Co, wp,
                       status, st);
    }
    return gemm(LoadGy2x2{gy, s, rows}, LoadRows{wp, 4 * s.Ci, 4 * s.Co}, EpiDx2x2{dx, dx32, mask, s, rows}, rows,
                4 * s.Ci, 4 * s.Co, 4 * s.Co, st);
}

// The 3 x 3 patch of position m for the four lanes of a quad (lane q holds
// taps q, q + 4 and, for q = 0, 8): each lane gathers at most three taps and
// the quad exchanges them by shuffles.  Called by whole warps.
__device__ __forceinline__ void conv1_patch_quad(const bf16 *__restrict__ x, const ConvShape &s, int m, int lane,
                                                 float xv[9]) {
    const int q = lane & 3;
    int b, oh, ow;
    pos_split(s, m, b, oh, ow);
    float mine[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int t = q + 4 * u, kh = (t * 11) >> 5, kw = t - 3 * kh;
        const int ih = 2 * oh - 1 + kh, iw = 2 * ow - 1 + kw;
        mine[u] = (t < 9 && ih >= 0 && ih < s.H && iw >= 0 && iw < s.W)
                      ? __bfloat162float(x[((size_t)b * s.H + ih) * s.W + iw])
                      : 0.f;
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) xv[t] = __shfl_sync(0xffffffffu, mine[t >> 2], (lane & ~3) | (t & 3));
}

// Per block: partial first-layer weight gradients over a grid-strided set of
// positions.  Four threads per position: thread q accumulates the 8 x 10
// products (channels 8 q .. 8 q + 7) x (9 taps and the bias's 1) of the
// positions it visits in registers (two positions per iteration, their loads
// in flight together); the block then sums the lanes that share
// q (shuffles) and the warps (shared memory) into part[block][320], ordered
// (co, tap) with the bias last.  k_conv1_wgrad_sum adds the blocks.
__global__ void __launch_bounds__(256, 2) k_conv1_wgrad_part(const bf16 *__restrict__ g, const bf16 *__restrict__ x,
                                                          ConvShape s, float *__restrict__ part) {
    __shared__ float red[8][320];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, q = lane & 3;
    float acc[8][10];
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int t = 0; t < 10; ++t) acc[c][t] = 0.f;
    const int64_t n = (int64_t)s.B * s.OH * s.OW * 4, stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count (the patch exchange is a whole-warp shuffle):
    // lanes past the end take position 0 with a zero gradient
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < n; base += 2 * stride) {
        // two positions per iteration (their loads in flight together)
        const int64_t e0 = base + lane, e1 = e0 + stride;
        const bool v0 = e0 < n, v1 = e1 < n;
        const int m0 = v0 ? (int)(e0 >> 2) : 0, m1 = v1 ? (int)(e1 >> 2) : 0;
        const uint4 u0 = v0 ? *reinterpret_cast<const uint4 *>(g + (size_t)m0 * 32 + 8 * q) : make_uint4(0, 0, 0, 0);
        const uint4 u1 = v1 ? *reinterpret_cast<const uint4 *>(g + (size_t)m1 * 32 + 8 * q) : make_uint4(0, 0, 0, 0);
        float xa[9], xb[9];
        conv1_patch_quad(x, s, m0, lane, xa);
        conv1_patch_quad(x, s, m1, lane, xb);
        const bf16 *h0 = reinterpret_cast<const bf16 *>(&u0), *h1 = reinterpret_cast<const bf16 *>(&u1);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float g0 = __bfloat162float(h0[c]), g1 = __bfloat162float(h1[c]);
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[c][t] = fmaf(g1, xb[t], fmaf(g0, xa[t], acc[c][t]));
            acc[c][9] += g0 + g1;
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int t = 0; t < 10; ++t) {
            float v = acc[c][t];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (lane < 4) red[warp][(8 * q + c) * 10 + t] = v;
        }
    __syncthreads();
    for (int o = tid; o < 320; o += blockDim.x) {
        float v = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) v += red[w8][o];
        part[(size_t)blockIdx.x * 320 + o] = v;
    }
}
// dw[co][tap] += sum over blocks of part[.][co * 10 + tap], db[co] likewise
// (tap 9): a warp per output, lanes striding over the blocks.
__global__ void k_conv1_wgrad_sum(const float *__restrict__ part, int nb, float *__restrict__ dw,
                                  float *__restrict__ db) {
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= 320) return;
    float v = 0.f;
    for (int b = lane; b < nb; b += 32) v += part[(size_t)b * 320 + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane) return;
    const int co = e / 10, k = e - 10 * co;
    if (k < 9) dw[co * 9 + k] += v;
    else db[co] += v;
}
constexpr int kConv1Blocks = 148 * 4;

cudaError_t conv_wgrad(const bf16 *gy, const bf16 *x, const ConvShape &s, float *dw, float *db, float *scratch,
                       unsigned *status, cudaStream_t st) {
    const int M = s.B * s.OH * s.OW, K = 9 * s.Ci;
    if (s.Ci == 1 && s.Co == 32) {
        const int nb = std::max(1, std::min(kConv1Blocks, (4 * M + 255) / 256));
        k_conv1_wgrad_part<<<nb, 256, 0, st>>>(gy, x, s, scratch);
        k_conv1_wgrad_sum<<<320 * 32 / 256, 256, 0, st>>>(scratch, nb, dw, db);
        return cudaGetLastError();
    }
    int bh, bb;
    const int xsw = s.Ci % 64 == 0 ? 128 : s.Ci == 32 ? 64 : 0;  // input boxes of xsw / 2 channels
    if (xsw && tile_rows(s, bh, bb, WG_K)) {
        // tensor-memory path: bias gradient by a column sum, dW by k_wgrad_tma
        CUtensorMap mG, mX;
        const uint64_t gd[2] = {(uint64_t)s.Co, (uint64_t)M}, gs[1] = {(uint64_t)s.Co * 2};
        const uint32_t gb[2] = {64, (uint32_t)WG_K}, ge[2] = {1, 1};
        const uint64_t xd[4] = {(uint64_t)s.Ci, (uint64_t)s.W, (uint64_t)s.H, (uint64_t)s.B};
        const uint64_t xs[3] = {(uint64_t)s.Ci * 2, (uint64_t)s.W * s.Ci * 2, (uint64_t)s.H * s.W * s.Ci * 2};
        const uint32_t xb[4] = {(uint32_t)(xsw / 2), (uint32_t)(2 * s.OW), (uint32_t)(2 * bh), (uint32_t)bb};
        const uint32_t xe[4] = {1, 2, 2, 1};
        if (encode_map(&mG, gy, 2, gd, gs, gb, ge) && encode_map(&mX, x, 4, xd, xs, xb, xe, xsw)) {
            if (db) {
                const int cb = (s.Co + 255) / 256;
                const int lpr = (s.Co < 256 && ilog2_exact(s.Co / 8) >= 0) ? s.Co / 8 : 32;
                const int rows_per_block = 8 * (32 / lpr) * 4;  // ~4 rows per lane
                const int bx = std::max(1, std::min((M + rows_per_block - 1) / rows_per_block, 4096));
                k_colsum_bf16_add<<<dim3(bx, cb), 256, 0, st>>>(gy, M, s.Co, lpr, db);
            }
            const int bn = (K % 128 == 0) ? 128 : 64, ntile = (K + bn - 1) / bn;
            const int nk = (M + WG_K - 1) / WG_K, tiles = ((s.Co + TC_M - 1) / TC_M) * ntile;
            const int splits = std::max(1, std::min(nk, (148 * 2 + tiles - 1) / tiles));
            const int steps = (nk + splits - 1) / splits;
            const dim3 grid((s.Co + TC_M - 1) / TC_M, ntile, (nk + steps - 1) / steps);
            const TmaA tx{TMA_CONV, ilog2_exact(s.Ci), ilog2_exact(s.OH * s.OW), ilog2_exact(s.OW)};
            cudaError_t e;
            if (bn == 128) {  // K % 128 == 0 implies Ci % 64 == 0 here (K = 9 Ci)
                e = cudaFuncSetAttribute(k_wgrad_tma<128, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcCfg<128>::SMEM);
                if (e) return e;
                k_wgrad_tma<128, 128><<<grid, TMA_THREADS, TcCfg<128>::SMEM, st>>>(mG, mX, tx, dw, s.Co, K, nk,
                                                                                   steps, status);
            } else if (xsw == 128) {
                e = cudaFuncSetAttribute(k_wgrad_tma<64, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcCfg<64>::SMEM);
                if (e) return e;
                k_wgrad_tma<64, 128><<<grid, TMA_THREADS, TcCfg<64>::SMEM, st>>>(mG, mX, tx, dw, s.Co, K, nk,
                                                                                 steps, status);
            } else {
                e = cudaFuncSetAttribute(k_wgrad_tma<64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcCfg<64>::SMEM);
                if (e) return e;
                k_wgrad_tma<64, 64><<<grid, TMA_THREADS, TcCfg<64>::SMEM, st>>>(mG, mX, tx, dw, s.Co, K, nk,
                                                                                steps, status);
            }
            return cudaGetLastError();
        }
    }
    // reduction over positions split so that the grid fills the GPU a few times
    const int tiles = ((s.Co + BM - 1) / BM) * ((K + 1 + BN - 1) / BN);
    const int splits = std::max(1, std::min((M + BK - 1) / BK, (148 * 4 + tiles - 1) / tiles));
    const int ksplit = (M + splits - 1) / splits;
    return gemm_t(LoadRowsT{gy, s.Co, s.Co}, LoadIm2colRowT{LoadIm2col{x, s, M, K}, K}, EpiWgrad{dw, db, s.Co, K},
                  s.Co, K + 1, M, ksplit, st);
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
    bf16 *wt = nullptr;    // sub-pixel weights scratch (input gradient)
    bf16 *act[kLayers + 1] = {};
    bf16 *gpre[kLayers + 1] = {};  // gradient at each conv output (after the ReLU mask)
    float *w1part = nullptr;  // first-layer weight-gradient block partials
    float *fc1part = nullptr; // fc1 split-K partial sums
    float *fc1wpart = nullptr;  // fc1 weight-gradient partial sums over batch splits
    float *h = nullptr, *z1 = nullptr, *a1 = nullptr, *out = nullptr, *dout = nullptr, *dz1 = nullptr, *dh = nullptr;
    unsigned *status = nullptr;  // device word: bit 4 = a tensor-memory GEMM's bounded wait ran out
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
                                     nullptr, n->status, st);
        if (e != cudaSuccess) return cuda_status(n, e, "conv forward");
    }
    const int F = layer_size(kLayers) * layer_size(kLayers) * kCh[kLayers], HD = F + kAux;
    k_flatten_concat<<<blocks_for((int64_t)B * HD), 256, 0, st>>>(n->act[kLayers], B, F, aux, n->h);
    sgemm(n->h, HD, 1, n->params + n->off_fc1w, HD, 1, B, kHidden, HD, EpiPart{n->fc1part, B, kHidden}, st,
          kFc1Splits);
    k_fc_finish<<<blocks_for((int64_t)B * kHidden), 256, 0, st>>>(n->fc1part, kFc1Splits, B, kHidden,
                                                                  n->params + n->off_fc1b, 1, n->z1, n->a1);
    sgemm(n->a1, kHidden, 1, n->params + n->off_fc2w, kHidden, 1, B, kOut, kHidden,
          EpiFc{n->out, nullptr, n->params + n->off_fc2b, B, kOut, 0}, st);
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
    size_t wt_max = 0;
    for (int l = 1; l < kLayers; ++l) {
        const size_t M = (size_t)B * layer_size(l + 1) * layer_size(l + 1);
        wt_max = std::max(wt_max, (size_t)16 * kCh[l] * kCh[l + 1]);
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
    if (!e) e = n->alloc(n->w1part, (size_t)kConv1Blocks * 320);
    if (!e) e = n->alloc(n->fc1part, (size_t)kFc1Splits * B * kHidden);
    if (!e) e = n->alloc(n->fc1wpart, (size_t)kFc1Splits * kHidden * HD);
    if (!e) e = n->alloc(n->h, (size_t)B * HD);
    if (!e) e = n->alloc(n->z1, (size_t)B * kHidden);
    if (!e) e = n->alloc(n->a1, (size_t)B * kHidden);
    if (!e) e = n->alloc(n->out, (size_t)B * kOut);
    if (!e) e = n->alloc(n->dout, (size_t)B * kOut);
    if (!e) e = n->alloc(n->dz1, (size_t)B * kHidden);
    if (!e) e = n->alloc(n->dh, (size_t)B * HD);
    if (!e) e = n->alloc(n->status, 1);
    if (!e) e = cudaMemset(n->status, 0, sizeof(unsigned));
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

gsvr_status gsvr_cnn_sync_status(gsvr_cnn *n) {
    unsigned word = 0;
    cudaError_t e;
    if (n) {
        DevGuard g(n->device);
        e = cudaStreamSynchronize(n->st);
        if (!e) e = cudaMemcpy(&word, n->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (!e) e = cudaMemset(n->status, 0, sizeof(unsigned));
    } else {
        e = cudaDeviceSynchronize();
        if (!e) e = cudaMemcpyFromSymbol(&word, g_tc_status, sizeof(unsigned));
        const unsigned zero = 0;
        if (!e) e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(unsigned));
    }
    if (e) return cuda_status(n, e, "sync status");
    if (word & 4u) return nfail(n, GSVR_ERR_TIMEOUT, "a tensor-memory GEMM's bounded wait ran out");
    return GSVR_OK;
}

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
    float *gr = n->grads;
    const float *p = n->params;
    sgemm(n->dout, 1, kOut, n->a1, 1, kHidden, kOut, kHidden, B, EpiF{gr + n->off_fc2w, nullptr, kOut, kHidden}, st);
    k_colsum_add<<<dim3(1, (B + 31) / 32), 256, 0, st>>>(n->dout, B, kOut, gr + n->off_fc2b);
    sgemm(n->dout, kOut, 1, p + n->off_fc2w, 1, kHidden, B, kHidden, kOut, EpiF{n->dz1, n->z1, B, kHidden}, st);
    {
        const int splits = std::max(1, std::min(kFc1Splits, B / 64));
        sgemm(n->dz1, 1, kHidden, n->h, 1, HD, kHidden, HD, B, EpiPart{n->fc1wpart, kHidden, HD}, st, splits);
        k_part_sum<<<blocks_for((int64_t)kHidden * HD), 256, 0, st>>>(n->fc1wpart, splits, (int64_t)kHidden * HD,
                                                                       gr + n->off_fc1w);
    }
    k_colsum_add<<<dim3((kHidden + 31) / 32, (B + 31) / 32), 256, 0, st>>>(n->dz1, B, kHidden, gr + n->off_fc1b);
    sgemm(n->dz1, kHidden, 1, p + n->off_fc1w, 1, HD, B, HD, kHidden, EpiF{n->dh, nullptr, B, HD}, st);
    k_flatten_grad<<<blocks_for((int64_t)B * F), 256, 0, st>>>(n->dh, B, F, HD, n->act[kLayers],
                                                               n->gpre[kLayers]);
    e = cudaGetLastError();
    if (e) return cuda_status(n, e, "head backward");
    for (int l = kLayers - 1; l >= 0; --l) {
        const ConvShape sh = conv_shape(B, layer_size(l), layer_size(l), kCh[l], kCh[l + 1]);
        e = conv_wgrad(n->gpre[l + 1], n->act[l], sh, n->grads + n->off_w[l], n->grads + n->off_b[l], n->w1part,
                       n->status, st);
        if (e) return cuda_status(n, e, "conv wgrad");
        if (l > 0) {
            e = conv_dgrad(n->gpre[l + 1], sh, n->wbf + n->off_w[l], n->wt, n->act[l], n->gpre[l], nullptr,
                           n->status, st);
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
        !aligned16(x) || !aligned16(w) || !aligned16(y) || (y32 && !aligned16(y32)) ||
        (int64_t)B * H * W > (1LL << 30))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad conv forward arguments");
    const ConvShape s = conv_shape(B, H, W, Ci, Co);
    if (Ci == 1 && !(Co == 32 && relu && !y32 && bias))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "one input channel: Co 32, ReLU, bias, no y32");
    return cuda_status(nullptr,
                       conv_forward(reinterpret_cast<const bf16 *>(x), s, reinterpret_cast<const bf16 *>(w), bias, relu,
                                    reinterpret_cast<bf16 *>(y), y32, tc_status_word(),
                                    static_cast<cudaStream_t>(stream)),
                       "conv forward");
}

gsvr_status gsvr_cnn_conv_dgrad(void *stream, const uint16_t *gy, int32_t B, int32_t H, int32_t W, int32_t Ci,
                                const uint16_t *w, int32_t Co, const uint16_t *mask, uint16_t *dx, float *dx32) {
    g_cnn_error.clear();
    if (!gy || !w || !dx || B < 1 || H < 1 || W < 1 || Ci < 8 || (Ci % 8) || Co < 8 || (Co % 8) ||
        !aligned16(gy) || !aligned16(w) || !aligned16(dx) || (dx32 && !aligned16(dx32)) ||
        (mask && !aligned16(mask)) || (int64_t)B * H * W > (1LL << 30))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad conv dgrad arguments (Ci, Co multiples of 8)");
    const ConvShape s = conv_shape(B, H, W, Ci, Co);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bf16 *wt = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&wt), sizeof(bf16) * 16 * Ci * Co, st);
    if (e) return cuda_status(nullptr, e, "scratch");
    e = conv_dgrad(reinterpret_cast<const bf16 *>(gy), s, reinterpret_cast<const bf16 *>(w), wt,
                   reinterpret_cast<const bf16 *>(mask), reinterpret_cast<bf16 *>(dx), dx32, tc_status_word(), st);
    cudaFreeAsync(wt, st);
    return cuda_status(nullptr, e, "conv dgrad");
}

gsvr_status gsvr_cnn_gemm(void *stream, const uint16_t *A, const uint16_t *B, int32_t M, int32_t N, int32_t K, float *C,
                          int32_t tensor_memory, unsigned *status) {
    g_cnn_error.clear();
    if (!A || !B || !C || M < 1 || N < 1 || K < 8 || (K % 8) || !aligned16(A) || !aligned16(B) || !aligned16(C) ||
        tensor_memory < 0 || tensor_memory > 2 || (tensor_memory && !status) || (int64_t)M * K > (1LL << 31) || (int64_t)N * K > (1LL << 31))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad gemm arguments (K a multiple of 8)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const LoadRows la{reinterpret_cast<const bf16 *>(A), M, K}, lb{reinterpret_cast<const bf16 *>(B), N, K};
    const EpiDense ep{C, M, N};
    cudaError_t e;
    if (tensor_memory == 1) {
        CUtensorMap mA, mB;
        if (!map_rows(&mA, reinterpret_cast<const bf16 *>(A), M, K, TC_M) ||
            !map_rows(&mB, reinterpret_cast<const bf16 *>(B), N, K, N <= 64 ? 64 : 128))
            return nfail(nullptr, GSVR_ERR_CUDA, "tensor map encoding failed");
        e = launch_tma(mA, mB, TmaA{TMA_ROWS, 0, 0, 0}, ep, M, N, K, status, st);
    } else if (tensor_memory == 2) {
        e = gemm_tc(la, lb, ep, M, N, K, B, status, st);
    } else {
        e = gemm(la, lb, ep, M, N, K, K, st);
    }
    return cuda_status(nullptr, e, "gemm");
}

gsvr_status gsvr_cnn_conv_wgrad(void *stream, const uint16_t *gy, const uint16_t *x, int32_t B, int32_t H, int32_t W,
                                int32_t Ci, int32_t Co, float *dw, float *db) {
    g_cnn_error.clear();
    if (!gy || !x || !dw || B < 1 || H < 1 || W < 1 || Ci < 1 || (Ci % 8 && Ci != 1) || Co < 8 || (Co % 8) ||
        (Ci == 1 && (Co != 32 || !db)) || !aligned16(gy) || !aligned16(x) || !aligned16(dw) ||
        (int64_t)B * H * W > (1LL << 30))
        return nfail(nullptr, GSVR_ERR_INVALID_ARG, "bad conv wgrad arguments (Co a multiple of 8)");
    const ConvShape s = conv_shape(B, H, W, Ci, Co);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *scratch = nullptr;
    if (Ci == 1) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), sizeof(float) * kConv1Blocks * 320, st);
        if (e) return cuda_status(nullptr, e, "scratch");
    }
    cudaError_t e = conv_wgrad(reinterpret_cast<const bf16 *>(gy), reinterpret_cast<const bf16 *>(x), s, dw, db,
                               scratch, tc_status_word(), st);
    if (scratch) cudaFreeAsync(scratch, st);
    return cuda_status(nullptr, e, "conv wgrad");
}

}  // extern "C"
