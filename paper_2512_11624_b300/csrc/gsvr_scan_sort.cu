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

// VEC: in and out are 16-byte aligned, so a thread's 8 items move as two
// 16-byte loads and stores (all but a ragged last group).
template <bool VEC>
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
    const int i0 = base + threadIdx.x * kScanItems;
    const bool whole = VEC && i0 + kScanItems <= n;
    int v[kScanItems];
    if (whole) {
        const int4 a = reinterpret_cast<const int4 *>(in + i0)[0], b = reinterpret_cast<const int4 *>(in + i0)[1];
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = i0 + k < n ? in[i0 + k] : 0;
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    int tot;
    int ex = block_excl_scan<kScanThreads>(s, tot) + bsum[blockIdx.x];
    int o[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        o[k] = ex;
        ex += v[k];
    }
    if (whole) {
        reinterpret_cast<int4 *>(out + i0)[0] = make_int4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<int4 *>(out + i0)[1] = make_int4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (i0 + k < n) out[i0 + k] = o[k];
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

// ------------------------------------------------------ tile-key radix sort
// One stable pass of the (tile, record) key sort with the value carried as a
// pair (record, emit index), so the sorted references need no gather.  The
// block's keys and values arrive by two 1-D bulk copies (TMA engine) into
// shared memory; ranking reads them from there, so no thread waits on DRAM
// between its keys.  FIRST: the values are built from key_rec (emit index =
// input position) instead of read.
template <int RADIX>
struct TileSortSmem {
    uint32_t key[kSortTile];                 // input keys, then the block's keys in digit order
    int2 val[kSortTile];                     // input values (FIRST: key_rec as int[kSortTile])
    unsigned short src[kSortTile];           // digit order -> input position in the block
    unsigned short cnt[kSortThreads / 32][RADIX];
    int dstart[RADIX];                       // block's start of each digit run
    int gbase[RADIX];                        // global position of the run minus dstart
    uint64_t bar;
};

template <bool FIRST, int RADIX>
__global__ void __launch_bounds__(kSortThreads, 3)
    k_tile_sort_scatter(const uint32_t *__restrict__ kin, const int2 *__restrict__ vin,
                        const int *__restrict__ key_rec, uint32_t *__restrict__ kout, int2 *__restrict__ vout,
                        const int *d_n, int n_max, int shift, const int *__restrict__ hist_scan, int nb,
                        unsigned *status) {
    constexpr int NW = kSortThreads / 32;
    constexpr int DPT = RADIX / kSortThreads;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileSortSmem<RADIX> &S = *reinterpret_cast<TileSortSmem<RADIX> *>(smem_raw);
    const int n = min(*d_n, n_max);
    const int base = blockIdx.x * kSortTile;
    if (base >= n) return;
    const int nk = min(kSortTile, n - base);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    int *skr = reinterpret_cast<int *>(S.val);
    // bulk parts (16-byte multiples; base is a multiple of kSortTile elements)
    const uint32_t kbytes = (uint32_t)(nk * 4) & ~15u;
    const uint32_t vbytes = FIRST ? ((uint32_t)(nk * 4) & ~15u) : ((uint32_t)(nk * 8) & ~15u);
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&S.bar, kbytes + vbytes);
        if (kbytes) bulk_g2s(S.key, kin + base, kbytes, &S.bar);
        if (vbytes) {
            if (FIRST) bulk_g2s(skr, key_rec + base, vbytes, &S.bar);
            else bulk_g2s(S.val, vin + base, vbytes, &S.bar);
        }
    }
    // meanwhile: this block's digit bases (strided in the digit-major scan)
    int gb[DPT];
#pragma unroll
    for (int k = 0; k < DPT; ++k) gb[k] = hist_scan[(tid * DPT + k) * nb + blockIdx.x];
    for (int d = lane; d < RADIX; d += 32) S.cnt[w][d] = 0;
    // the ragged tails the bulk copies leave (< 4 keys, < 4 or < 2 values)
    for (int e = (int)(kbytes / 4) + tid; e < nk; e += kSortThreads) S.key[e] = kin[base + e];
    if (FIRST)
        for (int e = (int)(vbytes / 4) + tid; e < nk; e += kSortThreads) skr[e] = key_rec[base + e];
    else
        for (int e = (int)(vbytes / 8) + tid; e < nk; e += kSortThreads) S.val[e] = vin[base + e];
    __syncthreads();  // barrier initialised (thread 0) before anyone polls it
    const bool ok = __syncthreads_and(mbar_wait_bounded(&S.bar, 0u, kWaitLimitNs));
    if (!ok) {  // (block-uniform) flag it, leave no copy in flight (bounded again), give up on the block
        if (tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            mbar_wait_bounded(&S.bar, 0u, kWaitLimitNs);
        }
        return;
    }
    // stable in-block ranks: warp w owns inputs w*512 .. w*512+511 in (round, lane) order
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[kSortItems];
    int rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int e = w * (32 * kSortItems) + r * 32 + lane;
        key[r] = e < nk ? S.key[e] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int e = w * (32 * kSortItems) + r * 32 + lane;
        const bool in = e < nk;
        const unsigned d = in ? ((key[r] >> shift) & (RADIX - 1u)) : (unsigned)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = 0;
        if (in) before = S.cnt[w][d];
        __syncwarp();
        if (in) {
            rank[r] = before + __popc(peers & lt);
            if ((peers & lt) == 0) S.cnt[w][d] = (unsigned short)(before + __popc(peers));
        } else {
            rank[r] = -1;
        }
        __syncwarp();
    }
    __syncthreads();
    {
        int runs[DPT], sum = 0;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            const int d = tid * DPT + k;
            int run = 0;
#pragma unroll
            for (int ww = 0; ww < NW; ++ww) {
                const int c = S.cnt[ww][d];
                S.cnt[ww][d] = (unsigned short)run;
                run += c;
            }
            runs[k] = run;
            sum += run;
        }
        int total;
        int start = block_excl_scan<kSortThreads>(sum, total);
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            S.dstart[tid * DPT + k] = start;
            S.gbase[tid * DPT + k] = gb[k] - start;
            start += runs[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (rank[r] < 0) continue;
        const unsigned d = (key[r] >> shift) & (RADIX - 1u);
        const int local = S.dstart[d] + S.cnt[w][d] + rank[r];
        S.key[local] = key[r];
        S.src[local] = (unsigned short)(w * (32 * kSortItems) + r * 32 + lane);
    }
    __syncthreads();
    // digit runs to their global ranges: consecutive threads, consecutive addresses
#pragma unroll 4
    for (int i = tid; i < nk; i += kSortThreads) {
        const uint32_t k = S.key[i];
        const int pos = S.gbase[(k >> shift) & (RADIX - 1u)] + i;
        const int e = S.src[i];
        const int2 v = FIRST ? make_int2(skr[e], base + e) : S.val[e];
        kout[pos] = k;
        vout[pos] = v;
    }
}

template <int RADIX>
__global__ void __launch_bounds__(kSortThreads) k_tile_sort_hist(const uint32_t *__restrict__ keys, const int *d_n,
                                                                 int n_max, int shift, int *hist, int nb) {
    __shared__ int cnt[RADIX];
    const int n = min(*d_n, n_max);
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    if (base < n) {
        const int nk = min(kSortTile, n - base);
        const int n4 = nk >> 2;  // whole 16-byte groups (keys + base is 16-byte aligned)
        const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + base);
        constexpr int G = kSortItems / 4;
        uint4 q[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = g * kSortThreads + threadIdx.x;
            q[g] = j < n4 ? k4[j] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g * kSortThreads + threadIdx.x >= n4) continue;
            atomicAdd(&cnt[(q[g].x >> shift) & (RADIX - 1u)], 1);
            atomicAdd(&cnt[(q[g].y >> shift) & (RADIX - 1u)], 1);
            atomicAdd(&cnt[(q[g].z >> shift) & (RADIX - 1u)], 1);
            atomicAdd(&cnt[(q[g].w >> shift) & (RADIX - 1u)], 1);
        }
        for (int e = 4 * n4 + threadIdx.x; e < nk; e += kSortThreads)
            atomicAdd(&cnt[(keys[base + e] >> shift) & (RADIX - 1u)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) hist[d * nb + blockIdx.x] = cnt[d];
}
}  // namespace

int scan_blocks(int n_max) { return n_max <= 0 ? 1 : (n_max + kScanTile - 1) / kScanTile; }

cudaError_t scan_exclusive(const int *in, int *out, const int *d_n, int n_static, int n_max, int *total_out,
                           const ScanScratch &s, cudaStream_t st) {
    const int nb = scan_blocks(n_max);
    if (nb > s.cap_blocks) return cudaErrorInvalidValue;
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, d_n, n_static, n_max, s.bsum);
    k_scan_bsum<<<1, 1024, 0, st>>>(s.bsum, nb);
    if ((((uintptr_t)in | (uintptr_t)out) & 15u) == 0)
        k_scan_down<true><<<nb, kScanThreads, 0, st>>>(in, out, d_n, n_static, n_max, s.bsum, nb, total_out);
    else
        k_scan_down<false><<<nb, kScanThreads, 0, st>>>(in, out, d_n, n_static, n_max, s.bsum, nb, total_out);
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

namespace {
template <bool FIRST, int RADIX>
cudaError_t launch_tile_sort_scatter(const uint32_t *kin, const int2 *vin, const int *key_rec, uint32_t *kout,
                                     int2 *vout, const int *d_n, int n_max, int shift, const int *hist, int nb,
                                     unsigned *status, cudaStream_t st) {
    constexpr size_t smem = sizeof(TileSortSmem<RADIX>);
    static int attr_dev = -1;  // the device whose attribute is set (one per process and instance)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(k_tile_sort_scatter<FIRST, RADIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    k_tile_sort_scatter<FIRST, RADIX><<<nb, kSortThreads, smem, st>>>(kin, vin, key_rec, kout, vout, d_n, n_max,
                                                                      shift, hist, nb, status);
    return cudaSuccess;
}
}  // namespace

cudaError_t sort_tile_keys(const uint32_t *keys, const int *key_rec, uint32_t *keys_out, int2 *tref, const int *d_n,
                           int n_max, int bits, const TileSortScratch &s, unsigned *status, cudaStream_t st) {
    if (n_max <= 0) return cudaSuccess;
    if (((uintptr_t)keys | (uintptr_t)key_rec | (uintptr_t)keys_out | (uintptr_t)tref |
         (uintptr_t)s.keys_alt | (uintptr_t)s.vals_alt) & 15u)
        return cudaErrorMisalignedAddress;  // bulk copies need 16-byte aligned buffers
    const int nb = sort_blocks(n_max);
    const int passes = bits <= 0 ? 1 : (bits + kSortDigitMax - 1) / kSortDigitMax;
    const int width = bits <= 0 ? 8 : std::max(1, (bits + passes - 1) / passes);
    const bool wide = width > 8;
    const int radix = wide ? 512 : 256;
    const uint32_t *ksrc = keys;
    const int2 *vsrc = nullptr;
    for (int p = 0; p < passes; ++p) {
        // the last pass lands in (keys_out, tref); earlier ones alternate with the scratch pair
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *kdst = to_out ? keys_out : s.keys_alt;
        int2 *vdst = to_out ? tref : s.vals_alt;
        const int shift = width * p;
        if (wide) k_tile_sort_hist<512><<<nb, kSortThreads, 0, st>>>(ksrc, d_n, n_max, shift, s.hist, nb);
        else k_tile_sort_hist<256><<<nb, kSortThreads, 0, st>>>(ksrc, d_n, n_max, shift, s.hist, nb);
        cudaError_t e = scan_exclusive(s.hist, s.hist, nullptr, radix * nb, radix * nb, nullptr, s.scan, st);
        if (e != cudaSuccess) return e;
        if (p == 0 && wide)
            e = launch_tile_sort_scatter<true, 512>(ksrc, vsrc, key_rec, kdst, vdst, d_n, n_max, shift, s.hist, nb,
                                                    status, st);
        else if (p == 0)
            e = launch_tile_sort_scatter<true, 256>(ksrc, vsrc, key_rec, kdst, vdst, d_n, n_max, shift, s.hist, nb,
                                                    status, st);
        else if (wide)
            e = launch_tile_sort_scatter<false, 512>(ksrc, vsrc, key_rec, kdst, vdst, d_n, n_max, shift, s.hist,
                                                     nb, status, st);
        else
            e = launch_tile_sort_scatter<false, 256>(ksrc, vsrc, key_rec, kdst, vdst, d_n, n_max, shift, s.hist,
                                                     nb, status, st);
        if (e != cudaSuccess) return e;
        note_launches(2);
        ksrc = kdst;
        vsrc = vdst;
    }
    return cudaGetLastError();
}

}  // namespace gsvr
