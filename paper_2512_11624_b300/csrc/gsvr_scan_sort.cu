// gsvr_scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort
// used by the binning pass ((tile, record) keys sorted by tile id).
//
// Both read their element count from device memory, so they run without a
// host round trip (grids are sized for the capacity; blocks past the count
// exit).  Radix sort: 8-bit digits; per pass an upsweep histogram per block,
// an exclusive scan of the digit-major histogram, and a stable scatter whose
// in-block ranks come from warp-level __match_any_sync over (warp, round, lane)
// order, so equal keys keep their input order.
#include <algorithm>

#include "gsvr_launch.cuh"

namespace gsvr {

namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = kScanTile / kScanThreads;  // 8

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int &total) {
    __shared__ int wsum[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = lane < NT / 32 ? wsum[lane] : 0;
        int xi = warp_incl_scan(x);
        if (lane < NT / 32) wsum[lane] = xi - x;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    int excl = inc - v + wsum[w];
    __shared__ int tot;
    if (threadIdx.x == NT - 1) tot = excl + v;
    __syncthreads();
    total = tot;
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *in, const int *d_n, int n_static,
                                                              int n_max, int *bsum) {
    const int n = d_n ? min(*d_n, n_max) : n_static;
    const int base = blockIdx.x * kScanTile;
    int s = 0;
    if (base < n) {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int idx = base + k * kScanThreads + threadIdx.x;
            if (idx < n) s += in[idx];
        }
    }
    int tot;
    block_excl_scan<kScanThreads>(s, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single block: exclusive scan of nb block sums in place; bsum[nb] = total.
__global__ void __launch_bounds__(1024) k_scan_bsum(int *bsum, int nb) {
    int carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int idx = base + threadIdx.x;
        int v = idx < nb ? bsum[idx] : 0;
        int tot;
        int ex = block_excl_scan<1024>(v, tot);
        if (idx < nb) bsum[idx] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int *in, int *out, const int *d_n,
                                                            int n_static, int n_max, const int *bsum, int nb,
                                                            int *total_out) {
    const int n = d_n ? min(*d_n, n_max) : n_static;
    const int base = blockIdx.x * kScanTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[n] = bsum[nb];
        if (total_out) *total_out = bsum[nb];
    }
    if (base >= n) return;
    // blocked arrangement: thread t owns items base + t*8 .. +7 (sequential order)
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + threadIdx.x * kScanItems + k;
        v[k] = idx < n ? in[idx] : 0;
        s += v[k];
    }
    int tot;
    int ex = block_excl_scan<kScanThreads>(s, tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + threadIdx.x * kScanItems + k;
        if (idx < n) out[idx] = ex;
        ex += v[k];
    }
}

// ---------------------------------------------------------------- radix sort
template <int RADIX>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *keys, const int *d_n, int n_max,
                                                             int shift, int *hist, int nb) {
    __shared__ int cnt[RADIX];
    const int n = min(*d_n, n_max);
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    if (base < n) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 4
        for (int r = 0; r < kSortItems; ++r) {
            int idx = base + w * (32 * kSortItems) + r * 32 + lane;
            if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & (RADIX - 1u)], 1);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) hist[d * nb + blockIdx.x] = cnt[d];
}

// GATHER: instead of the values, write tref[pos] = (key_rec[value], value): the
// record of the key and the key's emit index, in sorted (tile) order.
// The block first orders its tile by digit in shared memory (stable), then
// writes each digit's run to its global range with consecutive threads on
// consecutive addresses (coalesced stores).
template <bool GATHER, int RADIX>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t *kin, const uint32_t *vin,
                                                                uint32_t *kout, uint32_t *vout, const int *d_n,
                                                                int n_max, int shift, const int *hist_scan,
                                                                int nb, const int *key_rec, int2 *tref) {
    constexpr int NW = kSortThreads / 32;
    constexpr int DPT = RADIX / kSortThreads;  // digits per thread in the digit scans
    // per-warp digit counts fit 16 bits (a warp ranks 32 x kSortItems keys)
    __shared__ unsigned short cnt[NW][RADIX];
    __shared__ int dstart[RADIX];
    __shared__ uint32_t skey[kSortTile], sval[kSortTile];
    const int n = min(*d_n, n_max);
    const int base = blockIdx.x * kSortTile;
    if (base >= n) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < RADIX; d += 32) cnt[w][d] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[kSortItems], val[kSortItems];
    int rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int idx = base + w * (32 * kSortItems) + r * 32 + lane;
        const bool ok = idx < n;
        key[r] = ok ? kin[idx] : 0u;
        val[r] = ok ? (vin ? vin[idx] : (uint32_t)idx) : 0u;
        const unsigned d = ok ? ((key[r] >> shift) & (RADIX - 1u)) : (unsigned)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = 0;
        if (ok) before = cnt[w][d];
        __syncwarp();
        if (ok) {
            rank[r] = before + __popc(peers & lt);
            if ((peers & lt) == 0) cnt[w][d] = (unsigned short)(before + __popc(peers));
        } else {
            rank[r] = -1;
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then the block's digit starts
    // (thread t owns digits t * DPT .. t * DPT + DPT - 1)
    {
        int runs[DPT], sum = 0;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            const int d = threadIdx.x * DPT + k;
            int run = 0;
#pragma unroll
            for (int ww = 0; ww < NW; ++ww) {
                const int c = cnt[ww][d];
                cnt[ww][d] = (unsigned short)run;
                run += c;
            }
            runs[k] = run;
            sum += run;
        }
        int total;
        int start = block_excl_scan<kSortThreads>(sum, total);
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            dstart[threadIdx.x * DPT + k] = start;
            start += runs[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (rank[r] < 0) continue;
        const unsigned d = (key[r] >> shift) & (RADIX - 1u);
        const int local = dstart[d] + cnt[w][d] + rank[r];
        skey[local] = key[r];
        sval[local] = val[r];
    }
    __syncthreads();
    const int nb_keys = min(kSortTile, n - base);
    if (!GATHER) {
        for (int i = threadIdx.x; i < nb_keys; i += kSortThreads) {
            const uint32_t k = skey[i];
            const unsigned d = (k >> shift) & (RADIX - 1u);
            const int pos = hist_scan[d * nb + blockIdx.x] + (i - dstart[d]);
            kout[pos] = k;
            vout[pos] = sval[i];
        }
        return;
    }
    // gather: four independent key -> record lookups in flight per thread
    constexpr int G = 4;
    for (int i0 = threadIdx.x; i0 < nb_keys; i0 += G * kSortThreads) {
        uint32_t v[G];
        int kr[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int i = i0 + q * kSortThreads;
            v[q] = i < nb_keys ? sval[i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < G; ++q) kr[q] = i0 + q * kSortThreads < nb_keys ? key_rec[v[q]] : 0;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int i = i0 + q * kSortThreads;
            if (i >= nb_keys) continue;
            const uint32_t k = skey[i];
            const unsigned d = (k >> shift) & (RADIX - 1u);
            const int pos = hist_scan[d * nb + blockIdx.x] + (i - dstart[d]);
            kout[pos] = k;
            tref[pos] = make_int2(kr[q], (int)v[q]);
        }
    }
}
}  // namespace

int scan_blocks(int n_max) { return n_max <= 0 ? 1 : (n_max + kScanTile - 1) / kScanTile; }

cudaError_t scan_exclusive(const int *in, int *out, const int *d_n, int n_static, int n_max, int *total_out,
                           const ScanScratch &s, cudaStream_t st) {
    const int nb = scan_blocks(n_max);
    if (nb > s.cap_blocks) return cudaErrorInvalidValue;
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, d_n, n_static, n_max, s.bsum);
    k_scan_bsum<<<1, 1024, 0, st>>>(s.bsum, nb);
    k_scan_down<<<nb, kScanThreads, 0, st>>>(in, out, d_n, n_static, n_max, s.bsum, nb, total_out);
    note_launches(3);
    return cudaGetLastError();
}

int sort_blocks(int n_max) { return n_max <= 0 ? 1 : (n_max + kSortTile - 1) / kSortTile; }

size_t sort_hist_size(int n_max) { return (size_t)kSortRadixMax * (size_t)sort_blocks(n_max) + 1; }

cudaError_t radix_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                             uint32_t *vals_out, const int *d_n, int n_max, int bits, const SortScratch &s,
                             cudaStream_t st, const int *key_rec, int2 *tref) {
    const int nb = sort_blocks(n_max);
    // passes of equal digit width, at most 9 bits (512 bins): 16-bit keys take two
    // 8-bit passes, 17- and 18-bit keys two 9-bit passes
    const int passes = bits <= 0 ? 1 : (bits + kSortDigitMax - 1) / kSortDigitMax;
    const int width = bits <= 0 ? 8 : std::max(1, (bits + passes - 1) / passes);
    const bool wide = width > 8;
    const int radix = wide ? 512 : 256;
    const uint32_t *ksrc = keys_in;
    const uint32_t *vsrc = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *kdst = to_out ? keys_out : s.keys_alt;
        uint32_t *vdst = to_out ? vals_out : s.vals_alt;
        const int shift = width * p;
        if (wide) k_radix_hist<512><<<nb, kSortThreads, 0, st>>>(ksrc, d_n, n_max, shift, s.hist, nb);
        else k_radix_hist<256><<<nb, kSortThreads, 0, st>>>(ksrc, d_n, n_max, shift, s.hist, nb);
        cudaError_t e = scan_exclusive(s.hist, s.hist, nullptr, radix * nb, radix * nb, nullptr, s.scan, st);
        if (e != cudaSuccess) return e;
        const bool last = tref && p == passes - 1;
        if (last && wide)
            k_radix_scatter<true, 512><<<nb, kSortThreads, 0, st>>>(ksrc, vsrc, kdst, vdst, d_n, n_max, shift,
                                                                    s.hist, nb, key_rec, tref);
        else if (last)
            k_radix_scatter<true, 256><<<nb, kSortThreads, 0, st>>>(ksrc, vsrc, kdst, vdst, d_n, n_max, shift,
                                                                    s.hist, nb, key_rec, tref);
        else if (wide)
            k_radix_scatter<false, 512><<<nb, kSortThreads, 0, st>>>(ksrc, vsrc, kdst, vdst, d_n, n_max, shift,
                                                                     s.hist, nb, nullptr, nullptr);
        else
            k_radix_scatter<false, 256><<<nb, kSortThreads, 0, st>>>(ksrc, vsrc, kdst, vdst, d_n, n_max, shift,
                                                                     s.hist, nb, nullptr, nullptr);
        note_launches(2);
        ksrc = kdst;
        vsrc = vdst;
    }
    return cudaGetLastError();
}

}  // namespace gsvr
