// gsvr_metrics.cu -- image-quality metrics of a reconstructed volume against
// its ground truth on the same grid (Sec. 3, Table 1: PSNR, SSIM, NCC).
//
// X (reconstruction) and Y (reference) are float32 volumes of D x H x W voxels
// (x fastest); every metric is taken over the voxels of a mask.
//   PSNR = 10 log10(L^2 / MSE), L the data range;
//   NCC  = the Pearson correlation of X and Y;
//   SSIM (Wang et al. 2004, K1 = 0.01, K2 = 0.03) with the 11-tap Gaussian
//        window of standard deviation 1.5 voxels, in 3D the product window
//        11 x 11 x 11, kept to the grid and renormalised near its border; the
//        SSIM map is averaged over the masked voxels.
//
// The local moments mu_X, mu_Y, E[X^2], E[Y^2], E[XY] are three separable
// passes (x, y, z): the window is a product of per-axis taps, and the part of
// a box-shaped window that stays on a box-shaped grid is a product of per-axis
// intervals, so the renormalised 3D window is exactly the product of the
// per-axis renormalised windows.  The passes use taps normalised over the full
// window; the border renormalisation, the product of the per-axis in-grid tap
// sums, depends only on the output voxel's coordinates and is applied once in
// the last pass (it is 1 away from the border).  All sums are float64: the local variances
// E[X^2] - mu^2 are differences that cancel in flat regions, where float32
// would leave errors comparable to C2.  The masked sums of PSNR and NCC and
// the SSIM partial sums are reduced per block and then in one fixed order, so
// results do not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gsvr_launch.cuh"

namespace {

constexpr int kR = 5;              // window radius (11 taps)
constexpr int kTaps = 2 * kR + 1;
constexpr int kRowBlock = 128;     // x-pass outputs per block
constexpr int kThreads = 256;
constexpr int kSumBlocksMax = 148 * 8;
constexpr int kNSums = 8;          // n, Sx, Sy, Sxx, Syy, Sxy, Sdd, Sssim

struct Taps {
    double g[kTaps];  // exp(-o^2 / (2 sigma^2)), o = -kR .. kR, divided by their sum
};

// Sum of the taps whose offset keeps coordinate c inside [0, n): 1 unless c is
// within kR of either end.
__device__ __forceinline__ double in_grid_taps(const Taps &tp, int c, int n) {
    if (c >= kR && c + kR < n) return 1.0;
    double t = 0.0;
#pragma unroll
    for (int o = -kR; o <= kR; ++o)
        if (c + o >= 0 && c + o < n) t += tp.g[o + kR];
    return t;
}

// x pass: five moments of (X, Y) over the in-grid taps along x (not yet
// renormalised).  One block = kRowBlock outputs of one row; the row segment
// with its halo is staged once as the five per-voxel products (zeros off the
// grid).
__global__ void __launch_bounds__(kRowBlock) k_met_pass_x(const float *__restrict__ X, const float *__restrict__ Y,
                                                          int64_t rows, int W, int segs, Taps tp,
                                                          double *__restrict__ F, int64_t V) {
    __shared__ double s[5][kRowBlock + 2 * kR];
    const int64_t b = blockIdx.x;
    const int64_t row = b / segs;
    const int x0 = (int)(b % segs) * kRowBlock;
    if (row >= rows) return;
    const int64_t rb = row * (int64_t)W;
    for (int i = threadIdx.x; i < kRowBlock + 2 * kR; i += blockDim.x) {
        const int x = x0 - kR + i;
        double xv = 0.0, yv = 0.0;
        if (x >= 0 && x < W) {
            xv = (double)X[rb + x];
            yv = (double)Y[rb + x];
        }
        s[0][i] = xv;
        s[1][i] = yv;
        s[2][i] = xv * xv;
        s[3][i] = yv * yv;
        s[4][i] = xv * yv;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    // off-grid neighbours were staged as zeros, so every tap can be summed
    double a[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int o = -kR; o <= kR; ++o) {
        const double w = tp.g[o + kR];
        const int i = threadIdx.x + kR + o;
#pragma unroll
        for (int k = 0; k < 5; ++k) a[k] = fma(w, s[k][i], a[k]);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k * V + rb + x] = a[k];
}

// y or z pass over the five moment fields: along the axis of stride `stride`
// and extent `n` (interior outputs take every tap without a bounds test).  In
// the z pass (LAST) the sums are renormalised into the local moments; the SSIM
// map follows, is stored if asked, and its masked sum is reduced per block.
template <bool LAST>
__global__ void __launch_bounds__(kThreads) k_met_pass(const double *__restrict__ F, double *__restrict__ G, int64_t V,
                                                       int64_t stride, int n, int H, int W, Taps tp,
                                                       const uint8_t *__restrict__ mask, double C1, double C2,
                                                       double *__restrict__ map, double *__restrict__ part) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sval = 0.0;
    if (v < V) {
        const int c = (int)((v / stride) % n);
        double a[5] = {0, 0, 0, 0, 0};
        if (c >= kR && c + kR < n) {
#pragma unroll
            for (int o = -kR; o <= kR; ++o) {
                const double w = tp.g[o + kR];
                const int64_t u = v + (int64_t)o * stride;
#pragma unroll
                for (int k = 0; k < 5; ++k) a[k] = fma(w, __ldg(F + k * V + u), a[k]);
            }
        } else {
#pragma unroll
            for (int o = -kR; o <= kR; ++o) {
                if (c + o < 0 || c + o >= n) continue;
                const double w = tp.g[o + kR];
                const int64_t u = v + (int64_t)o * stride;
#pragma unroll
                for (int k = 0; k < 5; ++k) a[k] = fma(w, __ldg(F + k * V + u), a[k]);
            }
        }
        if (LAST) {
            // renormalise by the in-grid tap sums of the three axes
            const int x = (int)(v % W), y = (int)((v / W) % H);
            const double r = in_grid_taps(tp, x, W) * in_grid_taps(tp, y, H) * in_grid_taps(tp, c, n);
            if (r != 1.0) {
                const double inv = 1.0 / r;
#pragma unroll
                for (int k = 0; k < 5; ++k) a[k] *= inv;
            }
        }
        if (!LAST) {
#pragma unroll
            for (int k = 0; k < 5; ++k) G[k * V + v] = a[k];
        } else {
            const double mx = a[0], my = a[1];
            const double vx = a[2] - mx * mx, vy = a[3] - my * my, cxy = a[4] - mx * my;
            const double ssim = ((2.0 * mx * my + C1) * (2.0 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2));
            if (map) map[v] = ssim;
            if (!mask || mask[v]) sval = ssim;
        }
    }
    if (LAST) {
        __shared__ double red[kThreads / 32];
        for (int off = 16; off > 0; off >>= 1) sval += __shfl_xor_sync(0xffffffffu, sval, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sval;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            part[blockIdx.x] = t;
        }
    }
}

// Masked sums n, Sx, Sy, Sxx, Syy, Sxy, S(x-y)^2, one row of seven per block.
__global__ void __launch_bounds__(kThreads) k_met_sums(const float *__restrict__ X, const float *__restrict__ Y,
                                                       const uint8_t *__restrict__ mask, int64_t V,
                                                       double *__restrict__ part) {
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        if (mask && !mask[v]) continue;
        const double x = (double)X[v], y = (double)Y[v], d = x - y;
        a[0] += 1.0;
        a[1] += x;
        a[2] += y;
        a[3] += x * x;
        a[4] += y * y;
        a[5] += x * y;
        a[6] += d * d;
    }
    __shared__ double red[7][kThreads / 32];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double t = a[k];
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        part[(int64_t)blockIdx.x * 7 + threadIdx.x] = t;
    }
}

// One block: the partial sums in a fixed order, then the three metrics.
// out = {PSNR, SSIM, NCC, masked voxel count}.
__global__ void __launch_bounds__(kThreads) k_met_final(const double *__restrict__ sums, int nsb,
                                                        const double *__restrict__ ssim_part, int64_t nssb, double L,
                                                        double *__restrict__ out) {
    __shared__ double red[kNSums][kThreads];
    double a[kNSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nsb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 7; ++k) a[k] += sums[(int64_t)b * 7 + k];
    for (int64_t b = threadIdx.x; b < nssb; b += blockDim.x) a[7] += ssim_part[b];
#pragma unroll
    for (int k = 0; k < kNSums; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int k = 0; k < kNSums; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = red[0][0];
        const double sx = red[1][0], sy = red[2][0];
        const double vx = red[3][0] - sx * sx / n, vy = red[4][0] - sy * sy / n;
        const double cxy = red[5][0] - sx * sy / n;
        out[0] = 10.0 * log10(L * L / (red[6][0] / n));
        out[1] = red[7][0] / n;
        out[2] = cxy / sqrt(vx * vy);
        out[3] = n;
    }
}

// Scratch kept per device between calls (grown on demand, held until exit):
// a fresh allocation of 80 bytes per voxel would cost more than the passes.
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
Scratch g_scratch[kMaxDevices];

void set_msg(char *msg, int32_t len, const char *text) {
    if (msg && len > 0) {
        std::strncpy(msg, text, (size_t)len - 1);
        msg[len - 1] = '\0';
    }
}

}  // namespace

extern "C" gsvr_status gsvr_volume_metrics(int device, void *cuda_stream, int64_t D, int64_t H, int64_t W,
                                           const float *X, const float *Y, const uint8_t *mask, double data_range,
                                           double *out, double *ssim_map, char *msg, int32_t msg_len) {
    set_msg(msg, msg_len, "");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kMaxDevices) {
        cudaGetLastError();
        set_msg(msg, msg_len, "no such CUDA device");
        return GSVR_ERR_INVALID_ARG;
    }
    if (D <= 0 || H <= 0 || W <= 0 || W > (1 << 30) || H > (1 << 30) || D > (1 << 30) || !X || !Y || !out ||
        !(data_range > 0.0) || !std::isfinite(data_range)) {
        set_msg(msg, msg_len, "invalid argument");
        return GSVR_ERR_INVALID_ARG;
    }
    const int64_t V = D * H * W;
    if (V / D / H != W || V > ((int64_t)1 << 40)) {
        set_msg(msg, msg_len, "volume too large");
        return GSVR_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, device};
    cudaStream_t st = (cudaStream_t)cuda_stream;

    Taps tp;
    double gsum = 0.0;
    for (int o = -kR; o <= kR; ++o) gsum += (tp.g[o + kR] = std::exp(-0.5 * ((double)o / 1.5) * ((double)o / 1.5)));
    for (int o = -kR; o <= kR; ++o) tp.g[o + kR] /= gsum;
    const double C1 = (0.01 * data_range) * (0.01 * data_range);
    const double C2 = (0.03 * data_range) * (0.03 * data_range);

    const int64_t rows = D * H;
    const int segs = (int)((W + kRowBlock - 1) / kRowBlock);
    const int64_t xblocks = rows * segs;
    const int64_t vblocks = (V + kThreads - 1) / kThreads;
    const int nsb = (int)std::min<int64_t>(kSumBlocksMax, vblocks);
    if (xblocks > INT32_MAX || vblocks > INT32_MAX) {
        set_msg(msg, msg_len, "volume too large");
        return GSVR_ERR_INVALID_ARG;
    }
    cudaGetLastError();
    // scratch: two sets of five moment fields, the partial sums, the result
    const size_t fbytes = (size_t)5 * (size_t)V * sizeof(double);
    const size_t need = 2 * fbytes + ((size_t)nsb * 7 + (size_t)vblocks + 4) * sizeof(double);
    std::lock_guard<std::mutex> lock(g_scratch_mu);  // one call at a time uses the cached scratch
    Scratch &sc = g_scratch[device];
    if (sc.bytes < need) {
        if (sc.ptr) cudaFree(sc.ptr);
        sc.ptr = nullptr;
        sc.bytes = 0;
        if (cudaMalloc(&sc.ptr, need) != cudaSuccess) {
            cudaGetLastError();
            set_msg(msg, msg_len, "device allocation of the metric scratch failed");
            return GSVR_ERR_NOMEM;
        }
        sc.bytes = need;
    }
    double *F = static_cast<double *>(sc.ptr);
    double *G = F + 5 * V;
    double *sp = G + 5 * V;
    double *ssp = sp + (size_t)nsb * 7;
    double *dout = ssp + vblocks;
    double h[4] = {0, 0, 0, 0};
    k_met_sums<<<nsb, kThreads, 0, st>>>(X, Y, mask, V, sp);
    k_met_pass_x<<<(unsigned)xblocks, kRowBlock, 0, st>>>(X, Y, rows, (int)W, segs, tp, F, V);
    k_met_pass<false><<<(unsigned)vblocks, kThreads, 0, st>>>(F, G, V, W, (int)H, (int)H, (int)W, tp, nullptr, C1, C2,
                                                               nullptr, nullptr);
    k_met_pass<true><<<(unsigned)vblocks, kThreads, 0, st>>>(G, nullptr, V, H * W, (int)D, (int)H, (int)W, tp, mask,
                                                              C1, C2, ssim_map, ssp);
    k_met_final<<<1, kThreads, 0, st>>>(sp, nsb, ssp, vblocks, data_range, dout);
    gsvr::note_launches(5);
    cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, st);
    const cudaError_t e1 = cudaStreamSynchronize(st);
    const cudaError_t e2 = cudaGetLastError();
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        char b[160];
        std::snprintf(b, sizeof(b), "CUDA error: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        set_msg(msg, msg_len, b);
        return GSVR_ERR_CUDA;
    }
    for (int k = 0; k < 3; ++k) out[k] = h[k];
    if (h[3] < 1.0) {
        set_msg(msg, msg_len, "the mask selects no voxel");
        return GSVR_ERR_INVALID_ARG;
    }
    return GSVR_OK;
}
