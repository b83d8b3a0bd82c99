// gsvr_peaks.cu -- ALU throughput microbenchmarks used as roofline denominators
// for the tile kernels: float32 FFMA issue rate and MUFU ex2.approx rate of the
// whole GPU, measured with independent dependency chains in every thread of a
// grid that fills every SM (CUDA events around the launch).
#include <cuda_runtime.h>

#include "gsvr_launch.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_ffma(float *out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_ex2(float *out, int iters) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = gsvr::ex2_approx(-a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" gsvr_status gsvr_alu_peaks(int device, double *ffma_per_s, double *ex2_per_s, double *sm_count) {
    if (!ffma_per_s || !ex2_per_s) return GSVR_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    struct Restore {
        int prev;
        ~Restore() {
            if (prev >= 0) cudaSetDevice(prev);
        }
    } restore{prev};
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GSVR_ERR_INVALID_ARG;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    float *out = nullptr;
    if (cudaMalloc(&out, 256 * sizeof(float)) != cudaSuccess) return GSVR_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    double best_f = 0, best_e = 0;
    for (int rep = 0; rep < 3; ++rep) {
        float ms = 0;
        cudaEventRecord(e0);
        k_peak_ffma<<<blocks, threads>>>(out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best_f = fmax(best_f, (double)blocks * threads * iters * 16.0 * kChains / (ms * 1e-3));
        cudaEventRecord(e0);
        k_peak_ex2<<<blocks, threads>>>(out, iters / 4);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best_e = fmax(best_e, (double)blocks * threads * (iters / 4) * 16.0 * kChains / (ms * 1e-3));
    }
    gsvr::note_launches(6);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const cudaError_t err = cudaGetLastError();
    *ffma_per_s = best_f;
    *ex2_per_s = best_e;
    if (sm_count) *sm_count = nsm;
    return err == cudaSuccess ? GSVR_OK : GSVR_ERR_CUDA;
}

namespace {

__global__ void __launch_bounds__(256) k_peak_dfma(double *out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678) out[threadIdx.x] = s;
}

}  // namespace

extern "C" gsvr_status gsvr_fp64_peak(int device, double *dfma_per_s) {
    if (!dfma_per_s) return GSVR_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    struct Restore {
        int prev;
        ~Restore() {
            if (prev >= 0) cudaSetDevice(prev);
        }
    } restore{prev};
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GSVR_ERR_INVALID_ARG;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    double *out = nullptr;
    if (cudaMalloc(&out, 256 * sizeof(double)) != cudaSuccess) return GSVR_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8, threads = 256, iters = 64;
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        float ms = 0;
        cudaEventRecord(e0);
        k_peak_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best = fmax(best, (double)blocks * threads * iters * 16.0 * kChains / (ms * 1e-3));
    }
    gsvr::note_launches(3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const cudaError_t err = cudaGetLastError();
    *dfma_per_s = best;
    return err == cudaSuccess ? GSVR_OK : GSVR_ERR_CUDA;
}

namespace {

__global__ void __launch_bounds__(256) k_peak_ffma2(float *out, int iters, float b, float c) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(1e-3f * (float)(threadIdx.x + k), 2e-3f * (float)k);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = gsvr::f2_fma(a[k], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s == 12345.678f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" gsvr_status gsvr_ffma2_peak(int device, double *ffma2_per_s) {
    if (!ffma2_per_s) return GSVR_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    struct Restore {
        int prev;
        ~Restore() {
            if (prev >= 0) cudaSetDevice(prev);
        }
    } restore{prev};
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GSVR_ERR_INVALID_ARG;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    float *out = nullptr;
    if (cudaMalloc(&out, 256 * sizeof(float)) != cudaSuccess) return GSVR_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        float ms = 0;
        cudaEventRecord(e0);
        k_peak_ffma2<<<blocks, threads>>>(out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best = fmax(best, (double)blocks * threads * iters * 16.0 * kChains / (ms * 1e-3));
    }
    gsvr::note_launches(3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const cudaError_t err = cudaGetLastError();
    *ffma2_per_s = best;
    return err == cudaSuccess ? GSVR_OK : GSVR_ERR_CUDA;
}
