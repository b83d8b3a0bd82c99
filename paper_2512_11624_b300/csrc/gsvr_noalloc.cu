// gsvr_noalloc.cu -- gsvr_forward_noalloc: the forward pass for callers that
// cannot allocate device memory.
//
// Some host programs may not call cudaMalloc at all: code that runs inside a
// framework or plug-in whose device memory belongs to someone else, code under
// a strict memory budget or inside a region where allocation is forbidden.  For
// them this entry point runs the same kernels as gsvr_forward without a
// context: every intermediate buffer (slice frames, tile maps, sample lists,
// (slice, Gaussian) records, (tile, record) keys, sort buffers, per-tile
// partial losses) is carved from one file-scope device array of fixed size,
// kScratchBytes, that each GPU loading this library holds until the process
// exits.  The caller passes inputs and outputs; nothing is allocated on the
// device and no allocating library routine is called.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gsvr_launch.cuh"

using namespace gsvr;

namespace {

constexpr size_t kScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kTile = 16;
constexpr int kKeysPerRecord = 4;  // key capacity = 4 x record capacity
// Fixed scratch cost of one pixel: tile map, tile-order list and position,
// sample flags, flag offsets, sample list, residual (7 int32) and the mask byte.
constexpr size_t kPixelBytes = 7 * sizeof(int) + 1;
// Largest pixel count: the pixel arrays alone fill the scratch.
constexpr int64_t kMaxPixels = (int64_t)(kScratchBytes / kPixelBytes);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

void set_msg(char *msg, int32_t len, const char *text) {
    if (msg && len > 0) {
        std::strncpy(msg, text, (size_t)len - 1);
        msg[len - 1] = '\0';
    }
}

// Device address of g_scratch on the current device.  Looked up on every call
// (cheap once the library's module is loaded on the device), so a device reset
// or a re-created primary context never leaves a stale address behind.
cudaError_t scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carver {
    unsigned char *base;
    size_t off = 0, cap;
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += std::max<size_t>(n, 1) * sizeof(T);
        return p;
    }
    size_t used() const { return off; }
};

}  // namespace

extern "C" gsvr_status gsvr_forward_noalloc(int device, void *cuda_stream, int32_t n_stacks,
                                            const gsvr_stack_desc *stacks, int64_t N, const float *theta,
                                            const float *I, const int32_t *idx, int64_t n_idx, float cutoff_rel,
                                            int32_t norm_mode, float *pred, double *loss, char *msg,
                                            int32_t msg_len) {
    set_msg(msg, msg_len, "");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kMaxDevices) {
        cudaGetLastError();
        set_msg(msg, msg_len, "no such CUDA device");
        return GSVR_ERR_INVALID_ARG;
    }
    if (cutoff_rel == 0.f) cutoff_rel = 1e-7f;
    if (n_stacks <= 0 || !stacks || N < 0 || (N > 0 && !theta) || !I || !pred || !loss || n_idx < -1 ||
        (n_idx > 0 && !idx) || !(cutoff_rel > 0.f && cutoff_rel < 1.f) ||
        (norm_mode != GSVR_NORM_EXACT && norm_mode != GSVR_NORM_LITERAL)) {
        set_msg(msg, msg_len, "invalid argument");
        return GSVR_ERR_INVALID_ARG;
    }
    // geometry (host), as in gsvr_set_stacks: 16 x 16 pixel tiles
    std::vector<SliceDev> sl;
    std::vector<SliceStatic> ss;
    int64_t P = 0, T = 0;
    for (int s = 0; s < n_stacks; ++s) {
        const gsvr_stack_desc &d = stacks[s];
        bool ok = d.n_slices > 0 && d.H > 0 && d.W > 0 && d.H <= 65536 && d.W <= 65536 && d.dx > 0.f &&
                  d.dy > 0.f && d.thickness > 0.f;
        for (int e = 0; e < 9 && ok; ++e) ok = std::isfinite(d.R[e]);
        for (int e = 0; e < 3 && ok; ++e)
            ok = std::isfinite(d.origin[e]) && std::isfinite(d.fwhm[e]) && d.fwhm[e] >= 0.f;
        if (!ok) {
            set_msg(msg, msg_len, "invalid stack description");
            return GSVR_ERR_INVALID_ARG;
        }
        const int64_t tx = (d.W + kTile - 1) / kTile, ty = (d.H + kTile - 1) / kTile;
        const int64_t slice_px = (int64_t)d.H * d.W;
        if ((int64_t)d.n_slices * slice_px > kMaxPixels || P > kMaxPixels) {
            set_msg(msg, msg_len, "problem larger than the 32 MiB no-allocation scratch (pixel arrays)");
            return GSVR_ERR_INVALID_ARG;
        }
        for (int k = 0; k < d.n_slices; ++k) {
            SliceDev v{};
            SliceStatic st{};
            const double off = ((double)k - 0.5 * (d.n_slices - 1)) * (double)d.thickness;
            for (int e = 0; e < 9; ++e) st.R0[e] = d.R[e];
            for (int a = 0; a < 3; ++a) st.c0[a] = (double)d.origin[a] + off * (double)d.R[3 * a + 2];
            for (int a = 0; a < 3; ++a) {
                const double sg = (double)d.fwhm[a] / 2.355;
                v.var[a] = (float)(sg * sg);
            }
            v.dx = d.dx;
            v.dy = d.dy;
            v.cx0 = 0.5f * (float)(d.W - 1);
            v.cy0 = 0.5f * (float)(d.H - 1);
            v.H = d.H;
            v.W = d.W;
            v.tiles_x = (int)tx;
            v.tiles_y = (int)ty;
            v.tile_base = (int)T;
            v.pix_base = (int)P;
            v.stack = s;
            sl.push_back(v);
            ss.push_back(st);
            P += slice_px;
            T += tx * ty;
            if (P > kMaxPixels) {
                set_msg(msg, msg_len, "problem larger than the 32 MiB no-allocation scratch (pixel arrays)");
                return GSVR_ERR_INVALID_ARG;
            }
        }
    }
    const int M = (int)sl.size();
    if (n_idx > (int64_t)INT32_MAX / 2) {  // duplicates are allowed (counted once), as in gsvr_set_pixel_sample
        set_msg(msg, msg_len, "sample list longer than 2^30 entries");
        return GSVR_ERR_INVALID_ARG;
    }
    std::vector<int> tile_slice((size_t)T), pix_tile((size_t)P), tsp((size_t)P), tpos((size_t)P);
    {
        int64_t o = 0;
        for (int i = 0; i < M; ++i) {
            const SliceDev &v = sl[i];
            for (int ty = 0; ty < v.tiles_y; ++ty)
                for (int tx = 0; tx < v.tiles_x; ++tx) {
                    const int t = v.tile_base + ty * v.tiles_x + tx;
                    tile_slice[t] = i;
                    for (int a = ty * kTile; a < std::min(v.H, (ty + 1) * kTile); ++a)
                        for (int b = tx * kTile; b < std::min(v.W, (tx + 1) * kTile); ++b) {
                            const int p = v.pix_base + a * v.W + b;
                            pix_tile[p] = t;
                            tsp[o] = p;
                            tpos[p] = (int)o;
                            ++o;
                        }
                }
        }
    }

    // scratch layout: fixed part, then records and keys in the remaining space
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, device};
    void *base = nullptr;
    cudaGetLastError();
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        set_msg(msg, msg_len, "cudaGetSymbolAddress of the scratch array failed");
        return GSVR_ERR_CUDA;
    }
    Carver cv{reinterpret_cast<unsigned char *>(base), 0, kScratchBytes};
    SliceDev *d_sl = cv.take<SliceDev>(M);
    SliceStatic *d_ss = cv.take<SliceStatic>(M);
    int *d_tile_slice = cv.take<int>(T);
    int *d_pix_tile = cv.take<int>(P);
    int *d_tsp = cv.take<int>(P);
    int *d_tpos = cv.take<int>(P);
    uint8_t *d_mask = cv.take<uint8_t>(P);
    int *d_flags = cv.take<int>(P);
    int *d_flag_pos = cv.take<int>(P + 1);
    int *d_sampled = cv.take<int>(P);
    float *d_rbar = cv.take<float>(P);
    int *d_tps = cv.take<int>(T);
    int *d_tpe = cv.take<int>(T);
    int *d_trs = cv.take<int>(T);
    int *d_tre = cv.take<int>(T);
    double *d_tile_loss = cv.take<double>(T);
    double *d_subj_loss = cv.take<double>(1);
    float4 *d_gpre = cv.take<float4>(2 * N);
    int *d_rec_cnt = cv.take<int>(N + 1);
    int *d_rec_off = cv.take<int>(N + 1);
    unsigned *d_status = cv.take<unsigned>(1);
    Counters *d_cnt = cv.take<Counters>(1);
    const size_t fixed = cv.used();
    // per record: Rec + tile box + key count + key offset; per key: key, key_rec, sorted key and
    // value, two ping-pong words, (record, emit index) reference, backward moments (unused here), histogram share
    const size_t per_rec = sizeof(Rec) + 2 * sizeof(int2) + 3 * sizeof(int);
    const size_t per_key = 6 * sizeof(uint32_t) + sizeof(int2) + 1 + (kTile * kTile * sizeof(float)) / kItemRecs + 1;
    const size_t slack = 64 * 256 + 4096 * sizeof(int) + (size_t)(2 * T + 8) * (sizeof(int) + kTile * kTile * sizeof(float));
    if (fixed + slack + per_rec + kKeysPerRecord * per_key >= kScratchBytes) {
        set_msg(msg, msg_len,
                "problem larger than the 32 MiB no-allocation scratch (pixel, tile and Gaussian arrays leave "
                "no room for records)");
        return GSVR_ERR_INVALID_ARG;
    }
    const size_t room = kScratchBytes - fixed - slack;
    int cap_rec = (int)std::min<size_t>(room / (per_rec + kKeysPerRecord * per_key), (size_t)INT32_MAX / 8);
    int cap_keys = kKeysPerRecord * cap_rec;
    Rec *d_rec = cv.take<Rec>(cap_rec);
    int2 *d_rec_tiles = cv.take<int2>(cap_rec);
    int2 *d_cand = cv.take<int2>(cap_rec);
    int *d_rec_nkeys = cv.take<int>(cap_rec);
    unsigned *d_rec_mask = cv.take<unsigned>(cap_rec);
    int *d_key_off = cv.take<int>((size_t)cap_rec + 1);
    uint32_t *d_keys = cv.take<uint32_t>(cap_keys);
    int *d_key_rec = cv.take<int>(cap_keys);
    uint32_t *d_ks = cv.take<uint32_t>(cap_keys);
    uint32_t *d_vs = cv.take<uint32_t>(cap_keys);
    uint32_t *d_ka = cv.take<uint32_t>(cap_keys);
    uint32_t *d_va = cv.take<uint32_t>(cap_keys);
    int2 *d_tref = cv.take<int2>((size_t)cap_keys + 2);
    int *d_hist = cv.take<int>(sort_hist_size(cap_keys));
    const int cap_items = (int)(T + cap_keys / kItemRecs + 2);
    int *d_item_cnt = cv.take<int>(T + 1);
    int *d_item_first = cv.take<int>(T + 1);
    int *d_item_tile = cv.take<int>(cap_items);
    float *d_part = cv.take<float>((size_t)cap_items * kTile * kTile);
    const size_t scan_n = std::max<size_t>({(size_t)N + 1, (size_t)P + 1, (size_t)cap_rec + 1,
                                            sort_hist_size(cap_keys)});
    const int bsum_blocks = (int)((scan_n + kScanTile - 1) / kScanTile + 2);
    int *d_bsum = cv.take<int>((size_t)bsum_blocks + 1);
    if (cv.used() > kScratchBytes) {
        set_msg(msg, msg_len, "problem larger than the 32 MiB no-allocation scratch");
        return GSVR_ERR_INVALID_ARG;
    }
    const ScanScratch scs{d_bsum, bsum_blocks};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

#define NA_CK(call)                                                     \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            cudaGetLastError();                                         \
            set_msg(msg, msg_len, cudaGetErrorString(e_));              \
            return GSVR_ERR_CUDA;                                       \
        }                                                               \
    } while (0)

    // every call shares the array: upload the geometry, clear what starts at zero
    NA_CK(cudaMemcpyAsync(d_sl, sl.data(), sizeof(SliceDev) * M, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_ss, ss.data(), sizeof(SliceStatic) * M, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_tile_slice, tile_slice.data(), sizeof(int) * T, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_pix_tile, pix_tile.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_tsp, tsp.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_tpos, tpos.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(d_mask, 1, (size_t)P, st));
    NA_CK(cudaMemsetAsync(d_status, 0, sizeof(unsigned), st));
    NA_CK(cudaMemsetAsync(d_cnt, 0, sizeof(Counters), st));
    NA_CK(cudaMemsetAsync(d_tps, 0, sizeof(int) * T, st));
    NA_CK(cudaMemsetAsync(d_tpe, 0, sizeof(int) * T, st));
    NA_CK(cudaMemsetAsync(d_trs, 0, sizeof(int) * T, st));
    NA_CK(cudaMemsetAsync(d_tre, 0, sizeof(int) * T, st));

    // sample: the listed pixels (duplicates once) or every pixel, in tile order
    if (n_idx >= 0) {
        NA_CK(cudaMemsetAsync(d_flags, 0, sizeof(int) * P, st));
        launch_flags_from_list(idx, (int)n_idx, (int)P, d_mask, d_tpos, d_flags, d_status, st);
        NA_CK(scan_exclusive(d_flags, d_flag_pos, nullptr, (int)P, (int)P, &d_cnt->n_sampled, scs, st));
        launch_compact(d_flags, d_flag_pos, d_tsp, (int)P, d_sampled, st);
    } else {
        NA_CK(cudaMemcpyAsync(d_sampled, d_tsp, sizeof(int) * P, cudaMemcpyDeviceToDevice, st));
        launch_set_count(&d_cnt->n_sampled, (int)P, st);
    }
    launch_tile_px_ranges(d_sampled, &d_cnt->n_sampled, (int)P, d_pix_tile, d_tps, d_tpe, st);

    // forward: the same stages as gsvr_forward, at fixed capacity
    launch_gauss_prep(theta, (int)N, d_gpre, d_status, st);
    launch_pose_prep(theta + 11 * N, d_ss, d_sl, M, d_status, st);
    BinArgs b{};
    b.theta = theta;
    b.gpre = d_gpre;
    b.slices = d_sl;
    b.N = (int)N;
    b.M = M;
    b.rc2 = (float)(2.0 * std::log(1.0 / (double)cutoff_rel));
    b.norm_mode = norm_mode;
    b.tile_w = kTile;
    b.tile_h = kTile;
    b.qcut = (float)std::log2((double)cutoff_rel);
    b.tile_px_start = d_tps;
    b.tile_px_end = d_tpe;
    b.rec_cnt = d_rec_cnt;
    b.status = d_status;
    launch_cand_count(b, st);
    NA_CK(scan_exclusive(d_rec_cnt, d_rec_off, nullptr, (int)N, (int)N, &d_cnt->n_rec, scs, st));
    b.rec_off = d_rec_off;
    b.n_rec = &d_cnt->n_rec;
    b.cand = d_cand;
    b.rec = d_rec;
    b.rec_tiles = d_rec_tiles;
    b.rec_nkeys = d_rec_nkeys;
    b.rec_mask = d_rec_mask;
    b.cap_rec = cap_rec;
    launch_cand_emit(b, st);
    launch_records(b, cap_rec, st);
    NA_CK(scan_exclusive(d_rec_nkeys, d_key_off, &d_cnt->n_rec, 0, cap_rec, &d_cnt->n_keys, scs, st));
    KeyArgs k{};
    k.rec = d_rec;
    k.cand = d_cand;
    k.rec_tiles = d_rec_tiles;
    k.rec_nkeys = d_rec_nkeys;
    k.rec_mask = d_rec_mask;
    k.key_off = d_key_off;
    k.slices = d_sl;
    k.tile_px_start = d_tps;
    k.tile_px_end = d_tpe;
    k.n_rec = &d_cnt->n_rec;
    k.cap_rec = cap_rec;
    k.cap_keys = cap_keys;
    k.tile_w = kTile;
    k.tile_h = kTile;
    k.n_tiles = (int)T;
    k.qcut = b.qcut;
    k.keys = d_keys;
    k.key_rec = d_key_rec;
    k.status = d_status;
    launch_key_emit(k, cap_rec, st);
    int bits = 1;
    while ((1LL << bits) < T + 1) ++bits;
    const SortScratch sort_s{d_ka, d_va, d_hist, scs};
    NA_CK(radix_sort_pairs(d_keys, nullptr, d_ks, d_vs, &d_cnt->n_keys, cap_keys, bits, sort_s, st, d_key_rec,
                           d_tref));
    launch_tile_rec_ranges(d_ks, &d_cnt->n_keys, cap_keys, (int)T, d_trs, d_tre, st);
    launch_items(d_tps, d_tpe, d_trs, d_tre, (int)T, d_item_cnt, nullptr, nullptr, 0, 0, st);
    NA_CK(scan_exclusive(d_item_cnt, d_item_first, nullptr, (int)T, (int)T, &d_cnt->n_items, scs, st));
    launch_items(nullptr, nullptr, nullptr, nullptr, (int)T, nullptr, d_item_first, d_item_tile, cap_items, 1, st);
    EvalArgs e{};
    e.tref = d_tref;
    e.rec = d_rec;
    e.tile_rec_start = d_trs;
    e.tile_rec_end = d_tre;
    e.tile_px_start = d_tps;
    e.tile_px_end = d_tpe;
    e.tile_slice = d_tile_slice;
    e.slices = d_sl;
    e.sampled = d_sampled;
    e.n_sampled = &d_cnt->n_sampled;
    e.I_obs = I;
    e.pred = pred;
    e.rbar = d_rbar;
    e.tile_loss = d_tile_loss;
    e.counters = d_cnt;
    e.item_tile = d_item_tile;
    e.item_first = d_item_first;
    e.n_items = &d_cnt->n_items;
    e.part = d_part;
    e.cap_items = cap_items;
    e.tile_px = kTile * kTile;
    e.tile_w = kTile;
    e.tile_h = kTile;
    e.n_tiles = (int)T;
    e.status = d_status;
    e.qcut = b.qcut;
    launch_forward(e, st);
    launch_loss_reduce(d_tile_loss, (int)T, nullptr, 1, d_subj_loss, loss, d_status, st);
    NA_CK(cudaGetLastError());
    unsigned stt = 0;
    NA_CK(cudaMemcpyAsync(&stt, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (stt & ST_CAPACITY) {
        set_msg(msg, msg_len, "records or keys exceed the no-allocation scratch capacity");
        return GSVR_ERR_CAPACITY;
    }
    if (stt & ST_NONFINITE) {
        set_msg(msg, msg_len, "non-finite parameter, pose or loss");
        return GSVR_ERR_NONFINITE;
    }
    if (stt & ST_TIMEOUT) {
        set_msg(msg, msg_len, "a bounded device wait ran out");
        return GSVR_ERR_TIMEOUT;
    }
    if (stt & ST_INDEX) {
        set_msg(msg, msg_len, "pixel index out of range");
        return GSVR_ERR_INVALID_ARG;
    }
    return GSVR_OK;
}
