// gsvr_internal.cuh -- device data layout, PTX helpers and launcher declarations
// shared by the libgsvr.so translation units.  Nothing here is visible through
// the C ABI (include/gsvr.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gsvr.h"

namespace gsvr {

constexpr int kThreads = 128;     // threads of the tile kernels
constexpr int kItemRecs = 2 * kThreads;  // records per evaluation work item (one tile)
constexpr int kMaxTilePx = 1024;  // largest tile (32 x 32 pixels)
constexpr int kScanTile = 4096;   // items per block of the scans
constexpr int kSortThreads = 256; // 8 warps
constexpr int kSortItems = 16;    // keys per thread per radix pass (4096 per block)
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortDigitMax = 9;    // widest radix digit (bits) of one sort pass
constexpr int kSortRadixMax = 1 << kSortDigitMax;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s bound on any mbarrier wait

// Device status word bits (latched; read by gsvr_sync_status).
enum : unsigned { ST_CAPACITY = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u, ST_INDEX = 8u, ST_SHAPE = 16u };

// Per-slice frame and geometry.  The frame fields are rewritten from the pose
// every forward (Sec. 2.4: R_i = Rod(r) R0_i, t_i = Rod(r) c0_i + tau, computed in
// float64 per slice and stored as float32, plus float32 (hi, lo) pairs for the
// three projections that fix the record centres); the rest is fixed by the
// stack description.
struct SliceDev {
    float R[9];               // world-from-slice rotation, row-major (columns = slice axes)
    float t[3];               // world position of the slice centre
    float ux_h[3], ux_l[3];   // slice x axis / dx  (pixels per mm), hi + lo
    float uy_h[3], uy_l[3];   // slice y axis / dy
    float nz_h[3], nz_l[3];   // slice normal (mm per mm)
    float ox_h, ox_l;         // (x axis . t) / dx
    float oy_h, oy_l;         // (y axis . t) / dy
    float oz_h, oz_l;         // normal . t
    float var[3];             // Sigma_PSF diagonal (slice axes), mm^2
    float dx, dy;             // pixel spacing (mm)
    float cx0, cy0;           // (W-1)/2, (H-1)/2
    int H, W;
    int tiles_x, tiles_y;
    int tile_base;            // global id of the slice's first tile
    int pix_base;             // global index of the slice's first pixel
    int stack;
    int subject;              // reconstruction this slice belongs to (batched form)
    int pad_[2];
};

struct SliceStatic {
    double R0[9];   // nominal rotation (the stack's)
    double c0[3];   // nominal centre
};

// Device-side counts of the current forward.
struct Counters {
    int n_sampled;
    int n_rec;
    int n_keys;
    int n_items;
    unsigned long long pairs;  // pixel x record pairs visited by one evaluation pass
    unsigned long long step;   // device iteration counter (graph replay)
    int work_fwd, work_bwd;    // work-queue heads of the persistent evaluation kernels
    float adam_scal[4];        // Adam 1 / bias corrections and StepLR factor of a device-counted step
};

// A (slice, Gaussian) record: the 3D Gaussian conditioned on the slice plane
// (an exact identity: restricting exp(-1/2 v^T K^-1 v) to z = 0 gives a 2D
// Gaussian), in slice-centred pixel units, exponent pre-scaled by -1/2 log2(e):
//   f4[0] = (cb, ca, A, C2)   f4[1] = (B, w, j, i-or-key)
// value at pixel (b, a) = w * exp2(A db^2 + C2 db da + B da^2), db = b - cb, da = a - ca.
struct __align__(16) Rec {
    float4 a, b;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Packed two-wide float32 arithmetic (f32x2, sm_100 family) through the
// compiler's float2 builtins: each lane is the IEEE round-to-nearest scalar
// operation, two lanes per issue slot, and the compiler keeps the operands in
// register pairs (no packing moves around each instruction).
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`, giving up after `limit_ns` of wall time.
// The global timer is read once per 256 failed polls only: a read costs far
// more than a poll, and most waits end within a few polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    uint64_t t0 = 0;
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 0) {
            const uint64_t t = global_timer_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}

// ------------------------------------------------------------ launcher API
struct ScanScratch {
    int *bsum;   // >= blocks + 1 ints
    int cap_blocks;
};
// Exclusive scan of n int32 (n from *d_n when d_n != null, else n_static;
// n_max bounds the grid).  out[n] = total; *total_out = total when non-null.
cudaError_t scan_exclusive(const int *in, int *out, const int *d_n, int n_static, int n_max, int *total_out,
                           const ScanScratch &s, cudaStream_t st);
int scan_blocks(int n_max);

struct SortScratch {
    uint32_t *keys_alt, *vals_alt;  // ping-pong buffers (n_max each)
    int *hist;                      // 256 * blocks + 1
    ScanScratch scan;
};
int sort_blocks(int n_max);
// ints of the per-pass digit histogram (any digit width up to kSortDigitMax)
size_t sort_hist_size(int n_max);
// Stable LSD radix sort of n u32 keys (only the low `bits` bits are used, in
// ceil(bits / 9) passes of equal digit width) with
// u32 values; vals_in == null means values are the identity 0..n-1.  Result in
// keys_out / vals_out; when `tref` is given the last pass writes, instead of the
// values, tref[pos] = (key_rec[value], value).
cudaError_t radix_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                             uint32_t *vals_out, const int *d_n, int n_max, int bits, const SortScratch &s,
                             cudaStream_t st, const int *key_rec = nullptr, int2 *tref = nullptr);

struct TileSortScratch {
    uint32_t *keys_alt;  // n_max keys
    int2 *vals_alt;      // n_max (record, emit index) pairs
    int *hist;           // sort_hist_size(n_max)
    ScanScratch scan;
};
// Stable LSD radix sort of the n (= *d_n, at most n_max) tile keys in emit
// order (low `bits` bits, ceil(bits / 9) passes): keys_out[pos] = the sorted
// tile ids, tref[pos] = (key_rec[e], e) for the key from emit position e.  Every
// buffer 16-byte aligned (else cudaErrorMisalignedAddress); a bulk copy that
// does not complete within the wait bound sets ST_TIMEOUT in *status.
cudaError_t sort_tile_keys(const uint32_t *keys, const int *key_rec, uint32_t *keys_out, int2 *tref, const int *d_n,
                           int n_max, int bits, const TileSortScratch &s, unsigned *status, cudaStream_t st);

}  // namespace gsvr
