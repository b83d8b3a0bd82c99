// gsvr_api.cu -- the C ABI of libgsvr.so (declared in include/gsvr.h): context,
// device store (structure-of-arrays parameters, slice frames, pixel tiles),
// buffer management and the per-call orchestration of the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gsvr_launch.cuh"

using namespace gsvr;

namespace {

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    // Make room for `want` elements; contents are not kept.
    cudaError_t ensure(size_t want) {
        if (want <= n && p) return cudaSuccess;
        release();
        size_t bytes = std::max<size_t>(want, 1) * sizeof(T);
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), bytes);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = std::max<size_t>(want, 1);
        return cudaSuccess;
    }
};

thread_local std::string g_create_error;

}  // namespace

struct gsvr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    gsvr_config cfg{};
    std::string err;
    float rc2 = 0.f;
    int tile_w = 16, tile_h = 16;
    int fwd_pxr_req = 0, fwd_bps = 0, bwd_bps = 0, queue_order = 0;  // launch shape (gsvr_set_tiling)
    std::vector<gsvr_stack_desc> h_stack_desc;

    // geometry
    int n_stacks = 0, M = 0, n_tiles = 0, sort_bits = 1;
    int64_t P = 0;
    std::vector<SliceDev> h_slices;
    std::vector<SliceStatic> h_static;
    DBuf<SliceDev> d_slices;
    DBuf<SliceStatic> d_static;
    DBuf<int> d_tile_slice, d_pix_tile, d_pix_tpos, d_tile_sorted_pix;
    std::vector<int> h_tile_sorted_pix, h_tile_tpos_first, h_stack_nslices;

    // observations
    DBuf<float> d_I;
    DBuf<uint8_t> d_mask;
    DBuf<int> d_mask_tpos, d_mask_pix_sorted;
    DBuf<int> d_pix_mrank;  // per pixel: rank among the masked pixels in tile order (-1: unmasked)
    std::vector<int> h_mask_tpos;
    int n_mask = 0;

    // parameters
    int64_t N = 0;
    DBuf<float> d_theta, d_grad, d_m, d_v;
    DBuf<float4> d_gpre;
    DBuf<uint8_t> d_frozen;
    bool any_frozen = false;

    // sample
    DBuf<int> d_flags, d_flag_pos, d_sampled, d_tile_px_start, d_tile_px_end, d_idx;

    // binning
    DBuf<unsigned> d_rec_mask;
    DBuf<int> d_rec_cnt, d_rec_off, d_rec_nkeys, d_key_off, d_key_rec, d_tile_rec_start, d_tile_rec_end;
    DBuf<Rec> d_rec;
    DBuf<int2> d_tref;
    DBuf<int2> d_rec_tiles, d_cand;
    DBuf<uint32_t> d_keys, d_keys_sorted, d_keys_alt;
    DBuf<int2> d_vals_alt;
    DBuf<int> d_hist, d_scan_bsum;
    DBuf<unsigned> d_cand_mask;  // slab-test bits of the candidate count pass (single subject)
    DBuf<float4> d_mom;
    DBuf<int> d_item_cnt, d_item_first, d_item_tile;
    DBuf<uint32_t> d_item_key, d_item_key_sorted, d_item_order, d_item_key_alt, d_item_val_alt;
    DBuf<int> d_item_hist;
    DBuf<float> d_part;
    // objective (gsvr_set_objective): data term and scale regulariser
    int loss_kind = 0;
    float lambda_reg = 0.f, s_target = 1.6f;
    // per-slice outlier terms (gsvr_set_slice_weights): log sigma_i, log omega_i
    bool slw_on = false;
    float lr_slw_sig = 1e-3f, lr_slw_omg = 1e-2f;
    DBuf<float> d_slw, d_slw_grad, d_slw_m, d_slw_v;
    DBuf<double> d_slw_gacc, d_slw_tile;
    // content-adaptive initialisation scratch (gsvr_init_means)
    DBuf<int64_t> d_init_w, d_init_c, d_init_s;
    DBuf<float> d_init_pose, d_init_thick;
    // densification statistics and scratch (gsvr_densify_accumulate, gsvr_densify)
    DBuf<float4> d_dens_acc;          // per Gaussian: sum ||dL/dmu||, sum dL/dmu
    DBuf<int> d_dens_cnt, d_dens_nout, d_dens_off, d_dens_misc;
    DBuf<uint8_t> d_dens_kind;
    int64_t dens_n = -1;              // the N the statistics are sized for (-1: restart them)
    // normalised top-K form (gsvr_set_topk); K = 0: the plain sum
    int topk_K = 0, topk_refresh = 1;
    float topk_delta = 1e-8f, topk_per_cell = 16.f;
    int64_t topk_calls = 0, topk_n_dev = -1;  // topk_n_dev: the N held in d_topk_n
    DBuf<TopkGrid> d_topk_grid;
    DBuf<uint32_t> d_topk_keys, d_topk_keys_sorted, d_topk_gidx, d_topk_kalt, d_topk_valt;
    DBuf<int> d_topk_hist, d_topk_cstart, d_topk_cend, d_topk_nbr, d_topk_ncnt, d_topk_n;
    DBuf<float2> d_topk_pstat;
    DBuf<float4> d_topk_gm;
    DBuf<double> d_topk_loss_part;
    DBuf<float> d_topk_gacc;
    int cap_rec = 0, cap_keys = 0, cap_items = 0, grid_items = 0;
    int last_n_rec = 0, last_n_keys = 0;

    // outputs
    DBuf<float> d_pred, d_rbar;
    DBuf<int> d_tpos_s;    // tile-local (row << 8 | col) in sample order (written by the forward)
    DBuf<short2> d_row_rng;  // per tile row: sampled column range (written by the forward)
    DBuf<float> d_rbar_tile; // dense r_bar per tile pixel (built by the backward)
    DBuf<double> d_tile_loss, d_loss, d_pose_acc;
    DBuf<unsigned> d_status;
    DBuf<Counters> d_counters;

    bool have_stacks = false, have_obs = false, have_gauss = false, have_sample = false, fwd_valid = false;
    int64_t sample_total = 0;      // gsvr_set_sample_total: pixel weight 1 / sample_total (0: own sample size)
    int test_wait_forwards = 0;    // gsvr_test_wait_timeout: forwards left that run the hook
    int64_t test_wait_ns = 0;

    // subjects (batched form): stacks -> subject, contiguous Gaussian ranges
    int n_subj = 1;
    std::vector<int> h_stack_subject;   // per stack
    std::vector<int> h_subj_slice_first, h_subj_tile_first, h_subj_mask_first;
    std::vector<int64_t> h_subj_gauss_first;
    DBuf<int> d_gauss_subject, d_subj_slice_first, d_subj_tile_first, d_subj_mask_first, d_subj_out_first, d_subj_cnt;
    DBuf<double> d_subj_loss;
    DBuf<int> d_all_first;  // {0, n_mask}: the whole mask as one sampling range
    DBuf<int> d_single_out; // {0, n}: output offsets of a whole-mask sample
    int64_t single_out_n = -1, subj_out_n = -1, subj_out_total = 0;
    std::vector<uint8_t> h_subj_active;  // per subject (empty: every subject active)
    DBuf<uint8_t> d_subj_active;         // its device copy (read by the candidate pass)
    bool multi_gauss = false;

    // CUDA graph of one optimisation iteration
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool capturing = false;

    // stage timing (cfg.timing)
    struct Mark {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Mark> marks;
    cudaEvent_t open_ev[GSVR_N_STAGES] = {};
    double ms[GSVR_N_STAGES] = {};
    int64_t calls[GSVR_N_STAGES] = {};
    long long launches_at_reset = 0;
    DBuf<unsigned long long> d_pairs_total, d_bwd_pairs_total, d_useful;

    ~gsvr_ctx() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto &m : marks) {
            cudaEventDestroy(m.a);
            cudaEventDestroy(m.b);
        }
        for (auto e : ev_pool) cudaEventDestroy(e);
        for (auto e : open_ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

gsvr_status fail(gsvr_ctx *c, gsvr_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            cudaGetLastError();                                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? GSVR_ERR_NOMEM : GSVR_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                              \
        }                                                                                                 \
    } while (0)

bool finite_all(const float *v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

size_t scan_scratch_blocks(gsvr_ctx *ctx) {
    size_t n = std::max<size_t>({(size_t)ctx->N + 1, (size_t)ctx->P + 1, (size_t)ctx->cap_rec + 1,
                                 sort_hist_size(ctx->cap_keys),
                                 sort_hist_size((int)ctx->N),
                                 sort_hist_size(ctx->cap_items)});
    return (n + kScanTile - 1) / kScanTile + 2;
}

cudaError_t ensure_scan_scratch(gsvr_ctx *ctx) { return ctx->d_scan_bsum.ensure(scan_scratch_blocks(ctx) + 1); }

ScanScratch scan_scratch(gsvr_ctx *ctx) { return ScanScratch{ctx->d_scan_bsum.p, (int)ctx->d_scan_bsum.n - 1}; }

gsvr_status ensure_item_capacity(gsvr_ctx *ctx);

gsvr_status ensure_rec_capacity(gsvr_ctx *ctx, int64_t want) {
    if (want <= ctx->cap_rec && ctx->d_rec.p) return GSVR_OK;
    if (want > (int64_t)INT32_MAX - 16) return fail(ctx, GSVR_ERR_CAPACITY, "record count exceeds int32 range");
    const int cap = (int)std::min<int64_t>((int64_t)INT32_MAX - 16, std::max<int64_t>(want, 1024));
    CK(ctx->d_rec.ensure(cap));
    CK(ctx->d_rec_tiles.ensure(cap));
    CK(ctx->d_cand.ensure(cap));
    CK(ctx->d_rec_nkeys.ensure(cap));
    CK(ctx->d_rec_mask.ensure(cap));
    CK(ctx->d_key_off.ensure((size_t)cap + 1));
    ctx->cap_rec = cap;
    CK(ensure_scan_scratch(ctx));
    return GSVR_OK;
}

gsvr_status ensure_key_capacity(gsvr_ctx *ctx, int64_t want) {
    if (want <= ctx->cap_keys && ctx->d_keys.p) return GSVR_OK;
    if (want > (int64_t)INT32_MAX - 16) return fail(ctx, GSVR_ERR_CAPACITY, "key count exceeds int32 range");
    const int cap = (int)std::min<int64_t>((int64_t)INT32_MAX - 16, std::max<int64_t>(want, 4096));
    CK(ctx->d_keys.ensure(cap));
    CK(ctx->d_key_rec.ensure(cap));
    CK(ctx->d_keys_sorted.ensure(cap));
    CK(ctx->d_keys_alt.ensure(cap));
    CK(ctx->d_vals_alt.ensure(cap));
    CK(ctx->d_tref.ensure((size_t)cap + 2));
    CK(ctx->d_mom.ensure((size_t)cap * 2));
    CK(ctx->d_hist.ensure(sort_hist_size(cap)));
    ctx->cap_keys = cap;
    CK(ensure_scan_scratch(ctx));
    return ensure_item_capacity(ctx);
}

// Work items (<= kItemRecs records of one tile): at most one per tile plus one
// per kItemRecs keys.
gsvr_status ensure_item_capacity(gsvr_ctx *ctx) {
    const int64_t want = (int64_t)ctx->n_tiles + ctx->cap_keys / kItemRecs + 2;
    CK(ctx->d_item_cnt.ensure((size_t)ctx->n_tiles + 1));
    CK(ctx->d_item_first.ensure((size_t)ctx->n_tiles + 1));
    if (want > ctx->cap_items || !ctx->d_item_tile.p || ctx->d_part.n < (size_t)want * ctx->tile_w * ctx->tile_h) {
        CK(ctx->d_item_tile.ensure((size_t)want));
        CK(ctx->d_part.ensure((size_t)want * ctx->tile_w * ctx->tile_h));
        ctx->cap_items = (int)want;
    }
    if (ctx->queue_order && ctx->d_item_order.n < (size_t)ctx->cap_items) {
        const size_t n = (size_t)ctx->cap_items;
        CK(ctx->d_item_key.ensure(n));
        CK(ctx->d_item_key_sorted.ensure(n));
        CK(ctx->d_item_order.ensure(n));
        CK(ctx->d_item_key_alt.ensure(n));
        CK(ctx->d_item_val_alt.ensure(n));
        CK(ctx->d_item_hist.ensure(sort_hist_size(ctx->cap_items)));
    }
    CK(ensure_scan_scratch(ctx));
    return GSVR_OK;
}

EvalArgs eval_args(gsvr_ctx *ctx, int grid_items) {
    EvalArgs e{};
    e.tref = ctx->d_tref.p;
    e.rec = ctx->d_rec.p;
    e.tile_rec_start = ctx->d_tile_rec_start.p;
    e.tile_rec_end = ctx->d_tile_rec_end.p;
    e.tile_px_start = ctx->d_tile_px_start.p;
    e.tile_px_end = ctx->d_tile_px_end.p;
    e.tile_slice = ctx->d_tile_slice.p;
    e.slices = ctx->d_slices.p;
    e.sampled = ctx->d_sampled.p;
    e.n_sampled = &ctx->d_counters.p->n_sampled;
    e.I_obs = ctx->d_I.p;
    e.pred = ctx->d_pred.p;
    e.rbar = ctx->d_rbar.p;
    e.tpos_s = ctx->d_tpos_s.p;
    e.row_rng = ctx->d_row_rng.p;
    e.rbar_tile = ctx->d_rbar_tile.p;
    e.pix_tile = ctx->d_pix_tile.p;
    e.tile_loss = ctx->d_tile_loss.p;
    e.mom = ctx->d_mom.p;
    e.counters = ctx->d_counters.p;
    e.pairs_total = ctx->d_pairs_total.p;
    e.bwd_pairs_total = ctx->d_bwd_pairs_total.p;
    e.item_tile = ctx->d_item_tile.p;
    e.item_first = ctx->d_item_first.p;
    e.n_items = &ctx->d_counters.p->n_items;
    e.part = ctx->d_part.p;
    e.subj_cnt = ctx->n_subj > 1 ? ctx->d_subj_cnt.p : nullptr;
    e.cap_items = std::min(grid_items, ctx->cap_items);
    e.item_order = ctx->queue_order ? ctx->d_item_order.p : nullptr;
    e.fwd_pxr = ctx->fwd_pxr_req;
    e.fwd_bps = ctx->fwd_bps;
    e.bwd_bps = ctx->bwd_bps;
    e.tile_px = ctx->tile_w * ctx->tile_h;
    e.l1 = ctx->loss_kind;
    e.slw = ctx->slw_on ? ctx->d_slw.p : nullptr;
    e.slw_gacc = ctx->d_slw_gacc.p;
    e.slw_tile = ctx->d_slw_tile.p;
    e.M = ctx->M;
    e.tile_w = ctx->tile_w;
    e.tile_h = ctx->tile_h;
    e.n_tiles = ctx->n_tiles;
    e.status = ctx->d_status.p;
    e.n_weight = ctx->sample_total;
    e.qcut = (float)std::log2((double)ctx->cfg.cutoff_rel);
    return e;
}

// Subject tables on the device: slice / tile / mask ranges per subject and the
// subject of every Gaussian (only when more than one subject).
gsvr_status upload_subjects(gsvr_ctx *ctx) {
    const int n = ctx->n_subj;
    std::vector<int> slice_first(n + 1, 0), tile_first(n + 1, 0);
    {
        int sl = 0, k = 0;
        for (int st = 0; st < ctx->n_stacks; ++st) {
            const int sj = ctx->h_stack_subject.empty() ? 0 : ctx->h_stack_subject[st];
            while (k < sj) slice_first[++k] = sl;
            sl += ctx->h_stack_nslices[st];
        }
        while (k < n) slice_first[++k] = sl;
    }
    for (int k = 0; k <= n; ++k)
        tile_first[k] = slice_first[k] < ctx->M ? ctx->h_slices[slice_first[k]].tile_base : ctx->n_tiles;
    for (int i = 0; i < ctx->M; ++i) {
        int sj = 0;
        while (sj + 1 < n && slice_first[sj + 1] <= i) ++sj;
        ctx->h_slices[i].subject = sj;
    }
    ctx->h_subj_slice_first = slice_first;
    ctx->h_subj_tile_first = tile_first;
    CK(ctx->d_subj_slice_first.ensure(n + 1));
    CK(ctx->d_subj_tile_first.ensure(n + 1));
    CK(ctx->d_subj_mask_first.ensure(n + 1));
    CK(ctx->d_subj_out_first.ensure(n + 1));
    CK(ctx->d_subj_cnt.ensure(n));
    CK(ctx->d_subj_loss.ensure(n));
    CK(ctx->d_all_first.ensure(2));
    CK(ctx->d_single_out.ensure(2));
    ctx->single_out_n = -1;
    ctx->subj_out_n = -1;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->d_subj_slice_first.p, slice_first.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_subj_tile_first.p, tile_first.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_slices.p, ctx->h_slices.data(), sizeof(SliceDev) * ctx->M, cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->d_subj_loss.p, 0, sizeof(double) * n));
    return GSVR_OK;
}

// Mask ranges per subject (the masked pixels are in tile order, so subject-major).
gsvr_status upload_mask_ranges(gsvr_ctx *ctx, const std::vector<int> &mtp) {
    const int n = ctx->n_subj;
    std::vector<int> mf(n + 1, 0);
    size_t q = 0;
    for (int k = 0; k < n; ++k) {
        mf[k] = (int)q;
        const int tpos_end = ctx->h_subj_tile_first[k + 1] < ctx->n_tiles
                                 ? ctx->h_tile_tpos_first[ctx->h_subj_tile_first[k + 1]]
                                 : (int)ctx->P;
        while (q < mtp.size() && mtp[q] < tpos_end) ++q;
    }
    mf[n] = (int)mtp.size();
    ctx->h_subj_mask_first = mf;
    ctx->subj_out_n = -1;
    const int all[2] = {0, (int)mtp.size()};
    CK(cudaMemcpy(ctx->d_subj_mask_first.p, mf.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_all_first.p, all, sizeof(all), cudaMemcpyHostToDevice));
    return GSVR_OK;
}

// Tile ranges of the current sample (sampled pixels are in tile order).
gsvr_status finish_sample(gsvr_ctx *ctx) {
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(ctx->d_tile_px_start.p, 0, sizeof(int) * ctx->n_tiles, st));
    CK(cudaMemsetAsync(ctx->d_tile_px_end.p, 0, sizeof(int) * ctx->n_tiles, st));
    launch_tile_px_ranges(ctx->d_sampled.p, &ctx->d_counters.p->n_sampled, (int)ctx->P, ctx->d_pix_tile.p,
                          ctx->d_tile_px_start.p, ctx->d_tile_px_end.p, st);
    if (ctx->n_subj > 1)  // one subject: the weights read the total sample count
        launch_subject_counts(ctx->d_tile_px_start.p, ctx->d_tile_px_end.p, ctx->d_subj_tile_first.p, ctx->n_subj,
                              ctx->d_subj_cnt.p, st);
    CK(cudaGetLastError());
    ctx->have_sample = true;
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status sample_all(gsvr_ctx *ctx) {
    cudaStream_t st = ctx->stream;
    if (ctx->n_mask > 0)
        CK(cudaMemcpyAsync(ctx->d_sampled.p, ctx->d_mask_pix_sorted.p, sizeof(int) * ctx->n_mask,
                           cudaMemcpyDeviceToDevice, st));
    launch_set_count(&ctx->d_counters.p->n_sampled, ctx->n_mask, st);
    CK(cudaGetLastError());
    return finish_sample(ctx);
}

// Compact the flagged masked-rank positions into the sample (ranks follow the
// tile order, so the sample comes out in tile order).
gsvr_status compact_flags(gsvr_ctx *ctx) {
    cudaStream_t st = ctx->stream;
    if (ctx->n_mask > 0) {
        CK(scan_exclusive(ctx->d_flags.p, ctx->d_flag_pos.p, nullptr, ctx->n_mask, ctx->n_mask,
                          &ctx->d_counters.p->n_sampled, scan_scratch(ctx), st));
        launch_compact(ctx->d_flags.p, ctx->d_flag_pos.p, ctx->d_mask_pix_sorted.p, ctx->n_mask, ctx->d_sampled.p,
                       st);
    } else {
        launch_set_count(&ctx->d_counters.p->n_sampled, 0, st);
    }
    CK(cudaGetLastError());
    return finish_sample(ctx);
}

gsvr_status check_ctx(gsvr_ctx *ctx) { return ctx ? GSVR_OK : GSVR_ERR_INVALID_ARG; }

cudaEvent_t pooled_event(gsvr_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void fold_marks(gsvr_ctx *ctx) {
    for (auto &m : ctx->marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
            ctx->ms[m.stage] += t;
            ctx->calls[m.stage] += 1;
        }
        cudaGetLastError();
        ctx->ev_pool.push_back(m.a);
        ctx->ev_pool.push_back(m.b);
    }
    ctx->marks.clear();
}

// Stage timers: CUDA events on the context stream around each stage.
void stage_begin(gsvr_ctx *ctx, int stage) {
    if (!ctx->cfg.timing || ctx->capturing) return;
    cudaEvent_t e = pooled_event(ctx);
    if (!e) return;
    cudaEventRecord(e, ctx->stream);
    if (ctx->open_ev[stage]) ctx->ev_pool.push_back(ctx->open_ev[stage]);
    ctx->open_ev[stage] = e;
}
void stage_end(gsvr_ctx *ctx, int stage) {
    if (!ctx->cfg.timing || ctx->capturing || !ctx->open_ev[stage]) return;
    cudaEvent_t e = pooled_event(ctx);
    if (!e) return;
    cudaEventRecord(e, ctx->stream);
    ctx->marks.push_back({stage, ctx->open_ev[stage], e});
    ctx->open_ev[stage] = nullptr;
    if (ctx->marks.size() > 65536) {
        cudaStreamSynchronize(ctx->stream);
        fold_marks(ctx);
    }
}

}  // namespace

extern "C" {

int32_t gsvr_abi_version(void) { return GSVR_ABI_VERSION; }

const char *gsvr_last_error(gsvr_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

gsvr_status gsvr_create(gsvr_ctx **out, int device, void *cuda_stream, const gsvr_config *cfg) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return GSVR_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_create_error = "no such CUDA device";
        return GSVR_ERR_INVALID_ARG;
    }
    gsvr_config c{};
    if (cfg) c = *cfg;
    if (c.cutoff_rel == 0.f) c.cutoff_rel = 1e-7f;
    if (c.tile_w == 0) c.tile_w = 16;
    if (c.tile_h == 0) c.tile_h = 16;
    if (!(c.cutoff_rel > 0.f && c.cutoff_rel < 1.f) || (c.timing != 0 && c.timing != 1) || c.tile_w < 4 || c.tile_w > 32 || c.tile_h < 4 ||
        c.tile_h > 32 || (c.norm_mode != GSVR_NORM_EXACT && c.norm_mode != GSVR_NORM_LITERAL) ||
        c.cap_records < 0 || c.cap_keys < 0 || (c.fixed_capacity && (c.cap_records <= 0 || c.cap_keys <= 0))) {
        g_create_error = "invalid gsvr_config";
        return GSVR_ERR_INVALID_ARG;
    }
    gsvr_ctx *ctx = new (std::nothrow) gsvr_ctx();
    if (!ctx) return GSVR_ERR_NOMEM;
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    ctx->cfg = c;
    ctx->tile_w = c.tile_w;
    ctx->tile_h = c.tile_h;
    ctx->rc2 = (float)(2.0 * std::log(1.0 / (double)c.cutoff_rel));
    DeviceGuard g(device);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = ctx->d_status.ensure(1);
    if (e == cudaSuccess) e = ctx->d_counters.ensure(1);
    if (e == cudaSuccess) e = ctx->d_loss.ensure(1);
    if (e == cudaSuccess) e = ctx->d_pairs_total.ensure(1);
    if (e == cudaSuccess) e = ctx->d_bwd_pairs_total.ensure(1);
    if (e == cudaSuccess) e = ctx->d_useful.ensure(1);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_pairs_total.p, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_bwd_pairs_total.p, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status.p, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_counters.p, 0, sizeof(Counters));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_loss.p, 0, sizeof(double));
    if (e != cudaSuccess) {
        g_create_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        delete ctx;
        return GSVR_ERR_NOMEM;
    }
    *out = ctx;
    return GSVR_OK;
}

gsvr_status gsvr_destroy(gsvr_ctx *ctx) {
    if (!ctx) return GSVR_ERR_INVALID_ARG;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        delete ctx;
    }
    return GSVR_OK;
}

gsvr_status gsvr_set_stacks(gsvr_ctx *ctx, int32_t n_stacks, const gsvr_stack_desc *stacks) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (n_stacks <= 0 || !stacks) return fail(ctx, GSVR_ERR_INVALID_ARG, "need at least one stack");
    DeviceGuard g(ctx->device);
    ctx->slw_on = false;  // per-slice terms are sized by the slices: set them again
    const int tw = ctx->tile_w, th = ctx->tile_h;
    std::vector<SliceDev> sl;
    std::vector<SliceStatic> ss;
    int64_t P = 0, T = 0;
    for (int s = 0; s < n_stacks; ++s) {
        const gsvr_stack_desc &d = stacks[s];
        if (d.n_slices <= 0 || d.H <= 0 || d.W <= 0 || d.H > 65536 || d.W > 65536 || !(d.dx > 0.f) ||
            !(d.dy > 0.f) || !(d.thickness > 0.f) || !finite_all(d.R, 9) || !finite_all(d.origin, 3) ||
            !finite_all(d.fwhm, 3) || d.fwhm[0] < 0.f || d.fwhm[1] < 0.f || d.fwhm[2] < 0.f)
            return fail(ctx, GSVR_ERR_INVALID_ARG, "invalid stack description " + std::to_string(s));
        const int tx = (d.W + tw - 1) / tw, ty = (d.H + th - 1) / th;
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
            v.tiles_x = tx;
            v.tiles_y = ty;
            v.tile_base = (int)T;
            v.pix_base = (int)P;
            v.stack = s;
            P += (int64_t)d.H * d.W;
            T += (int64_t)tx * ty;
            if (P >= (int64_t)INT32_MAX / 2 || T >= (int64_t)INT32_MAX / 2)
                return fail(ctx, GSVR_ERR_INVALID_ARG, "too many pixels or tiles");
            sl.push_back(v);
            ss.push_back(st);
        }
    }
    const int M = (int)sl.size();
    // static pixel / tile maps: tile order = slice, tile row, tile col, row-major inside the tile
    std::vector<int> tile_slice((size_t)T), pix_tile((size_t)P), tsp((size_t)P), tpos((size_t)P);
    std::vector<int> tile_tpos_first((size_t)T);
    int64_t o = 0;
    for (int i = 0; i < M; ++i) {
        const SliceDev &v = sl[i];
        for (int ty = 0; ty < v.tiles_y; ++ty)
            for (int tx = 0; tx < v.tiles_x; ++tx) {
                const int t = v.tile_base + ty * v.tiles_x + tx;
                tile_slice[t] = i;
                tile_tpos_first[t] = (int)o;
                for (int a = ty * th; a < std::min(v.H, (ty + 1) * th); ++a)
                    for (int b = tx * tw; b < std::min(v.W, (tx + 1) * tw); ++b) {
                        const int p = v.pix_base + a * v.W + b;
                        pix_tile[p] = t;
                        tsp[o] = p;
                        tpos[p] = (int)o;
                        ++o;
                    }
            }
    }
    ctx->have_stacks = ctx->have_obs = ctx->have_sample = ctx->fwd_valid = false;
    ctx->n_stacks = n_stacks;
    ctx->M = M;
    ctx->P = P;
    ctx->n_tiles = (int)T;
    int bits = 1;
    while ((1LL << bits) < T + 1) ++bits;  // tile ids and the sentinel T
    ctx->sort_bits = bits;
    ctx->h_slices = sl;
    ctx->h_static = ss;
    ctx->h_stack_desc.assign(stacks, stacks + n_stacks);
    ctx->h_tile_sorted_pix = tsp;
    ctx->h_tile_tpos_first = tile_tpos_first;
    ctx->h_stack_nslices.assign(n_stacks, 0);
    for (int st2 = 0; st2 < n_stacks; ++st2) ctx->h_stack_nslices[st2] = stacks[st2].n_slices;
    ctx->n_subj = 1;
    ctx->h_subj_active.clear();
    ctx->h_stack_subject.assign(n_stacks, 0);
    ctx->multi_gauss = false;
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    CK(ctx->d_slices.ensure(M));
    CK(ctx->d_static.ensure(M));
    CK(ctx->d_tile_slice.ensure(T));
    CK(ctx->d_pix_tile.ensure(P));
    CK(ctx->d_pix_tpos.ensure(P));
    CK(ctx->d_tile_sorted_pix.ensure(P));
    CK(cudaMemcpy(ctx->d_slices.p, sl.data(), sizeof(SliceDev) * M, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_static.p, ss.data(), sizeof(SliceStatic) * M, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tile_slice.p, tile_slice.data(), sizeof(int) * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_pix_tile.p, pix_tile.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_pix_tpos.p, tpos.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tile_sorted_pix.p, tsp.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(ctx->d_I.ensure(P));
    CK(ctx->d_mask.ensure(P));
    CK(ctx->d_flags.ensure(P));
    CK(ctx->d_flag_pos.ensure(P + 1));
    CK(ctx->d_sampled.ensure(P));
    CK(ctx->d_pred.ensure(P));
    CK(ctx->d_rbar.ensure(P));
    CK(ctx->d_tpos_s.ensure(P));
    CK(ctx->d_row_rng.ensure((size_t)std::max(T, (int64_t)1) * ctx->tile_h));
    CK(ctx->d_rbar_tile.ensure((size_t)std::max(T, (int64_t)1) * ctx->tile_h * ctx->tile_w));
    CK(ctx->d_tile_px_start.ensure(T));
    CK(ctx->d_tile_px_end.ensure(T));
    CK(ctx->d_tile_rec_start.ensure(T));
    CK(ctx->d_tile_rec_end.ensure(T));
    CK(ctx->d_tile_loss.ensure(T));
    CK(ctx->d_pose_acc.ensure((size_t)M * 12));
    CK(ctx->d_frozen.ensure(M));
    CK(cudaMemset(ctx->d_frozen.p, 0, M));
    CK(cudaMemset(ctx->d_pred.p, 0, sizeof(float) * P));
    CK(cudaMemset(ctx->d_rbar.p, 0, sizeof(float) * P));
    ctx->any_frozen = false;
    CK(ensure_scan_scratch(ctx));
    {
        gsvr_status su = upload_subjects(ctx);
        if (su) return su;
    }
    // parameters sized for a different M are dropped
    if (ctx->have_gauss && ctx->d_theta.n != (size_t)(11 * ctx->N + 6 * M)) ctx->have_gauss = false;
    ctx->have_stacks = true;
    return GSVR_OK;
}

gsvr_status gsvr_set_observations(gsvr_ctx *ctx, const float *I, const uint8_t *mask, int32_t mem) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_stacks) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_stacks first");
    if (!I || (mem != GSVR_MEM_HOST && mem != GSVR_MEM_DEVICE))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad observation pointer or mem kind");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int64_t P = ctx->P;
    const cudaMemcpyKind kind = mem == GSVR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(ctx->d_I.p, I, sizeof(float) * P, kind, st));
    std::vector<uint8_t> hm((size_t)P, 1);
    if (mask) {
        if (mem == GSVR_MEM_HOST) memcpy(hm.data(), mask, (size_t)P);
        else CK(cudaMemcpyAsync(hm.data(), mask, (size_t)P, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (auto &v : hm) v = v ? 1 : 0;
    CK(cudaMemcpy(ctx->d_mask.p, hm.data(), (size_t)P, cudaMemcpyHostToDevice));
    std::vector<int> mtp, mps;
    mtp.reserve((size_t)P);
    for (int64_t t = 0; t < P; ++t) {
        const int p = ctx->h_tile_sorted_pix[(size_t)t];
        if (hm[(size_t)p]) {
            mtp.push_back((int)t);
            mps.push_back(p);
        }
    }
    ctx->n_mask = (int)mtp.size();
    {
        std::vector<int> mrank((size_t)P, -1);
        for (size_t q = 0; q < mps.size(); ++q) mrank[(size_t)mps[q]] = (int)q;
        CK(ctx->d_pix_mrank.ensure((size_t)P));
        CK(cudaMemcpy(ctx->d_pix_mrank.p, mrank.data(), sizeof(int) * (size_t)P, cudaMemcpyHostToDevice));
    }
    CK(ctx->d_mask_tpos.ensure(mtp.size()));
    CK(ctx->d_mask_pix_sorted.ensure(mps.size()));
    if (!mtp.empty()) {
        CK(cudaMemcpy(ctx->d_mask_tpos.p, mtp.data(), sizeof(int) * mtp.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_mask_pix_sorted.p, mps.data(), sizeof(int) * mps.size(), cudaMemcpyHostToDevice));
    }
    ctx->h_mask_tpos = mtp;
    {
        gsvr_status sm = upload_mask_ranges(ctx, mtp);
        if (sm) return sm;
    }
    ctx->have_obs = true;
    return sample_all(ctx);
}

// Record and key capacities for N Gaussians (the configured ones in
// fixed-capacity mode, else at least 8 records per Gaussian) and the scan
// scratch they imply.
gsvr_status gauss_capacities(gsvr_ctx *ctx, int64_t N) {
    if (ctx->cfg.fixed_capacity) {
        gsvr_status s = ensure_rec_capacity(ctx, ctx->cfg.cap_records);
        if (s) return s;
        s = ensure_key_capacity(ctx, ctx->cfg.cap_keys);
        if (s) return s;
    } else {
        const int64_t want_r = ctx->cfg.cap_records > 0 ? ctx->cfg.cap_records : std::max<int64_t>(4096, 8 * N);
        const int64_t want_k = ctx->cfg.cap_keys > 0 ? ctx->cfg.cap_keys : 4 * want_r;
        gsvr_status s = ensure_rec_capacity(ctx, std::max<int64_t>(ctx->cap_rec, want_r));
        if (s) return s;
        s = ensure_key_capacity(ctx, std::max<int64_t>(ctx->cap_keys, want_k));
        if (s) return s;
    }
    CK(ensure_scan_scratch(ctx));
    return GSVR_OK;
}

gsvr_status gsvr_set_gaussians(gsvr_ctx *ctx, int64_t N, const float *theta_g, int32_t mem) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_stacks) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_stacks first");
    if (N < 0 || N > (1LL << 26) || (N > 0 && !theta_g) || (mem != GSVR_MEM_HOST && mem != GSVR_MEM_DEVICE))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad Gaussian count, pointer or mem kind");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int M = ctx->M;
    const size_t np = (size_t)(11 * N + 6 * M);
    std::vector<float> pose((size_t)6 * M, 0.f);
    const bool keep_pose = ctx->have_gauss && ctx->d_theta.p && ctx->d_theta.n >= (size_t)(11 * ctx->N + 6 * M);
    std::vector<float> mv_pose((size_t)12 * M, 0.f);
    if (keep_pose && M > 0) {
        CK(cudaMemcpyAsync(pose.data(), ctx->d_theta.p + 11 * ctx->N, sizeof(float) * 6 * M, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaMemcpyAsync(mv_pose.data(), ctx->d_m.p + 11 * ctx->N, sizeof(float) * 6 * M, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaMemcpyAsync(mv_pose.data() + 6 * M, ctx->d_v.p + 11 * ctx->N, sizeof(float) * 6 * M,
                           cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    if (ctx->d_theta.n != np || !ctx->d_theta.p) {
        ctx->d_theta.release();
        ctx->d_grad.release();
        ctx->d_m.release();
        ctx->d_v.release();
    }
    CK(ctx->d_theta.ensure(np));
    CK(ctx->d_grad.ensure(np));
    CK(ctx->d_m.ensure(np));
    CK(ctx->d_v.ensure(np));
    CK(ctx->d_gpre.ensure((size_t)2 * N));
    CK(ctx->d_rec_cnt.ensure((size_t)N + 1));
    CK(ctx->d_rec_off.ensure((size_t)N + 1));
    ctx->N = N;
    if (N > 0)
        CK(cudaMemcpyAsync(ctx->d_theta.p, theta_g, sizeof(float) * 11 * N,
                           mem == GSVR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    if (M > 0) {
        CK(cudaMemcpyAsync(ctx->d_theta.p + 11 * N, pose.data(), sizeof(float) * 6 * M, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_m.p + 11 * N, mv_pose.data(), sizeof(float) * 6 * M, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_v.p + 11 * N, mv_pose.data() + 6 * M, sizeof(float) * 6 * M,
                           cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(ctx->d_grad.p, 0, sizeof(float) * np, st));
    if (N > 0) {
        CK(cudaMemsetAsync(ctx->d_m.p, 0, sizeof(float) * 11 * N, st));
        CK(cudaMemsetAsync(ctx->d_v.p, 0, sizeof(float) * 11 * N, st));
    }
    if (gsvr_status s = gauss_capacities(ctx, N)) return s;
    ctx->have_gauss = true;
    ctx->fwd_valid = false;
    ctx->dens_n = -1;  // densification statistics restart
    return GSVR_OK;
}

gsvr_status gsvr_set_poses(gsvr_ctx *ctx, const float *pose, int32_t mem) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_gaussians first");
    if (!pose || (mem != GSVR_MEM_HOST && mem != GSVR_MEM_DEVICE))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad pose pointer or mem kind");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int M = ctx->M;
    if (M > 0) {
        CK(cudaMemcpyAsync(ctx->d_theta.p + 11 * ctx->N, pose, sizeof(float) * 6 * M,
                           mem == GSVR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(ctx->d_m.p + 11 * ctx->N, 0, sizeof(float) * 6 * M, st));
        CK(cudaMemsetAsync(ctx->d_v.p + 11 * ctx->N, 0, sizeof(float) * 6 * M, st));
    }
    if (mem == GSVR_MEM_HOST) CK(cudaStreamSynchronize(st));
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status gsvr_reserve(gsvr_ctx *ctx, int64_t cap_records, int64_t cap_keys) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (cap_records < 0 || cap_keys < 0) return fail(ctx, GSVR_ERR_INVALID_ARG, "negative capacity");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_reserve during graph capture");
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    if (cap_records > ctx->cap_rec || cap_keys > ctx->cap_keys) {
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->graph) cudaGraphDestroy(ctx->graph);
        ctx->graph_exec = nullptr;
        ctx->graph = nullptr;
    }
    gsvr_status s = ensure_rec_capacity(ctx, std::max<int64_t>(cap_records, ctx->cap_rec));
    if (!s) s = ensure_key_capacity(ctx, std::max<int64_t>(cap_keys, ctx->cap_keys));
    if (s) return s;
    ctx->cfg.cap_records = std::max<int64_t>(ctx->cfg.cap_records, cap_records);
    ctx->cfg.cap_keys = std::max<int64_t>(ctx->cfg.cap_keys, cap_keys);
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status gsvr_set_frozen(gsvr_ctx *ctx, const uint8_t *frozen) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_stacks) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_stacks first");
    DeviceGuard g(ctx->device);
    std::vector<uint8_t> f((size_t)ctx->M, 0);
    bool any = false;
    if (frozen)
        for (int i = 0; i < ctx->M; ++i) {
            f[i] = frozen[i] ? 1 : 0;
            any = any || f[i];
        }
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->d_frozen.p, f.data(), (size_t)ctx->M, cudaMemcpyHostToDevice));
    ctx->any_frozen = any;
    return GSVR_OK;
}

gsvr_status gsvr_set_pixel_sample(gsvr_ctx *ctx, const int32_t *idx, int64_t n, int32_t mem) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_observations first");
    if (n < 0) {
        DeviceGuard g(ctx->device);
        return sample_all(ctx);
    }
    if ((n > 0 && !idx) || n > (int64_t)INT32_MAX / 2 || (mem != GSVR_MEM_HOST && mem != GSVR_MEM_DEVICE))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad sample pointer, size or mem kind");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int32_t *didx = idx;
    if (mem == GSVR_MEM_HOST && n > 0) {  // (indices are range-checked on the device, as device lists are)
        CK(ctx->d_idx.ensure((size_t)n));
        CK(cudaMemcpyAsync(ctx->d_idx.p, idx, sizeof(int) * n, cudaMemcpyHostToDevice, st));
        didx = ctx->d_idx.p;
    }
    CK(cudaMemsetAsync(ctx->d_flags.p, 0, sizeof(int) * ctx->n_mask, st));
    launch_flags_from_list_rank(didx, (int)n, (int)ctx->P, ctx->d_pix_mrank.p, ctx->d_flags.p, ctx->d_status.p,
                                st);
    CK(cudaGetLastError());
    return compact_flags(ctx);
}

// Flags from the device sampler over `ranges` (n_ranges mask ranges, out_first on the device).
gsvr_status sample_ranges(gsvr_ctx *ctx, int n_ranges, const int *mask_first, const int *out_first, int n_out,
                          uint64_t step, const unsigned long long *d_step) {
    cudaStream_t st = ctx->stream;
    stage_begin(ctx, GSVR_STAGE_SAMPLE);
    CK(cudaMemsetAsync(ctx->d_flags.p, 0, sizeof(int) * ctx->n_mask, st));
    launch_sample_flags(n_ranges, mask_first, out_first, n_out, ctx->cfg.seed, step, d_step, nullptr,
                        ctx->d_flags.p, st);
    CK(cudaGetLastError());
    gsvr_status s = compact_flags(ctx);
    stage_end(ctx, GSVR_STAGE_SAMPLE);
    return s;
}

gsvr_status gsvr_sample_pixels(gsvr_ctx *ctx, int64_t n, uint64_t step) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_observations first");
    if (n < 0 || n > ctx->n_mask) return fail(ctx, GSVR_ERR_INVALID_ARG, "sample larger than the masked pixels");
    DeviceGuard g(ctx->device);
    if (ctx->single_out_n != n) {  // offsets uploaded once per sample size
        const int out[2] = {0, (int)n};
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMemcpy(ctx->d_single_out.p, out, sizeof(out), cudaMemcpyHostToDevice));
        ctx->single_out_n = n;
    }
    return sample_ranges(ctx, 1, ctx->d_all_first.p, ctx->d_single_out.p, (int)n, step, nullptr);
}

// Per-subject output offsets of a sample of n pixels per subject (fewer where a
// subject has fewer masked pixels); uploads them and returns the total.
int64_t subject_out_first(gsvr_ctx *ctx, int64_t n) {
    if (ctx->subj_out_n == n) return ctx->subj_out_total;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    std::vector<int> of(ctx->n_subj + 1, 0);
    for (int k = 0; k < ctx->n_subj; ++k) {
        const int64_t avail = ctx->h_subj_mask_first[k + 1] - ctx->h_subj_mask_first[k];
        const bool on = ctx->h_subj_active.empty() || ctx->h_subj_active[(size_t)k];
        of[k + 1] = of[k] + (on ? (int)std::min<int64_t>(n, avail) : 0);
    }
    if (cudaMemcpy(ctx->d_subj_out_first.p, of.data(), sizeof(int) * of.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    ctx->subj_out_n = n;
    ctx->subj_out_total = of[ctx->n_subj];
    return of[ctx->n_subj];
}

gsvr_status gsvr_sample_pixels_subjects(gsvr_ctx *ctx, int64_t n_per_subject, uint64_t step) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_observations first");
    if (n_per_subject < 0) return fail(ctx, GSVR_ERR_INVALID_ARG, "negative sample size");
    DeviceGuard g(ctx->device);
    const int64_t tot = subject_out_first(ctx, n_per_subject);
    if (tot < 0) return fail(ctx, GSVR_ERR_CUDA, "upload of the sample offsets failed");
    return sample_ranges(ctx, ctx->n_subj, ctx->d_subj_mask_first.p, ctx->d_subj_out_first.p, (int)tot, step,
                         nullptr);
}

gsvr_status gsvr_set_subject_active(gsvr_ctx *ctx, const uint8_t *active) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss || !ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "set stacks, observations, Gaussians first");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_subject_active during graph capture");
    const int n = ctx->n_subj;
    std::vector<uint8_t> next((size_t)n, 1);
    if (active) {
        bool any = false;
        for (int k = 0; k < n; ++k) {
            next[(size_t)k] = active[k] ? 1 : 0;
            any = any || next[(size_t)k];
        }
        if (!any) return fail(ctx, GSVR_ERR_INVALID_ARG, "at least one subject must stay active");
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const std::vector<uint8_t> prev = ctx->h_subj_active.empty() ? std::vector<uint8_t>((size_t)n, 1)
                                                                 : ctx->h_subj_active;
    const int64_t N = ctx->N;
    for (int k = 0; k < n; ++k) {
        if (!prev[(size_t)k] || next[(size_t)k]) continue;
        // a subject leaving the sample: its Adam moments restart at zero, so the
        // zero gradient it now receives leaves its parameters where they are
        const int64_t g0 = n > 1 ? ctx->h_subj_gauss_first[(size_t)k] : 0;
        const int64_t g1 = n > 1 ? ctx->h_subj_gauss_first[(size_t)k + 1] : N;
        for (int c = 0; c < 11 && g1 > g0; ++c) {
            CK(cudaMemsetAsync(ctx->d_m.p + (size_t)c * N + g0, 0, sizeof(float) * (size_t)(g1 - g0), st));
            CK(cudaMemsetAsync(ctx->d_v.p + (size_t)c * N + g0, 0, sizeof(float) * (size_t)(g1 - g0), st));
        }
        const int s0 = n > 1 ? ctx->h_subj_slice_first[(size_t)k] : 0;
        const int s1 = n > 1 ? ctx->h_subj_slice_first[(size_t)k + 1] : ctx->M;
        if (s1 > s0) {
            CK(cudaMemsetAsync(ctx->d_m.p + 11 * N + 6 * (int64_t)s0, 0, sizeof(float) * 6 * (size_t)(s1 - s0), st));
            CK(cudaMemsetAsync(ctx->d_v.p + 11 * N + 6 * (int64_t)s0, 0, sizeof(float) * 6 * (size_t)(s1 - s0), st));
        }
    }
    ctx->h_subj_active = next;
    CK(ctx->d_subj_active.ensure((size_t)n));
    CK(cudaMemcpyAsync(ctx->d_subj_active.p, next.data(), (size_t)n, cudaMemcpyHostToDevice, st));
    ctx->subj_out_n = -1;  // per-subject sample offsets are recomputed
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    ctx->fwd_valid = false;
    CK(cudaStreamSynchronize(st));
    return GSVR_OK;
}

gsvr_status gsvr_set_subjects(gsvr_ctx *ctx, int32_t n, const int32_t *stack_subject, const int64_t *gauss_count) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss || !ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "set stacks, observations, Gaussians first");
    if (n < 1 || n > 65536 || (n > 1 && (!stack_subject || !gauss_count)))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad subject count or tables");
    std::vector<int> ss(ctx->n_stacks, 0);
    std::vector<int64_t> gf(n + 1, 0);
    if (n > 1) {
        int prev = 0;
        for (int k = 0; k < ctx->n_stacks; ++k) {
            ss[k] = stack_subject[k];
            if (ss[k] < prev || ss[k] > prev + 1 || ss[k] >= n)
                return fail(ctx, GSVR_ERR_INVALID_ARG, "stack subjects must be 0..n-1, contiguous, in order");
            prev = ss[k];
        }
        if (prev != n - 1) return fail(ctx, GSVR_ERR_INVALID_ARG, "every subject needs a stack");
        for (int k = 0; k < n; ++k) {
            if (gauss_count[k] < 0) return fail(ctx, GSVR_ERR_INVALID_ARG, "negative Gaussian count");
            gf[k + 1] = gf[k] + gauss_count[k];
        }
        if (gf[n] != ctx->N) return fail(ctx, GSVR_ERR_INVALID_ARG, "Gaussian counts must add up to N");
    } else {
        gf[1] = ctx->N;
    }
    DeviceGuard g(ctx->device);
    ctx->n_subj = n;
    ctx->h_subj_active.clear();
    ctx->h_stack_subject = ss;
    ctx->h_subj_gauss_first = gf;
    {
        gsvr_status su = upload_subjects(ctx);
        if (su) return su;
        su = upload_mask_ranges(ctx, ctx->h_mask_tpos);
        if (su) return su;
    }
    ctx->multi_gauss = n > 1;
    if (n > 1) {
        std::vector<int> gs((size_t)ctx->N);
        for (int k = 0; k < n; ++k)
            for (int64_t j = gf[k]; j < gf[k + 1]; ++j) gs[(size_t)j] = k;
        CK(ctx->d_gauss_subject.ensure((size_t)std::max<int64_t>(ctx->N, 1)));
        if (ctx->N > 0)
            CK(cudaMemcpy(ctx->d_gauss_subject.p, gs.data(), sizeof(int) * gs.size(), cudaMemcpyHostToDevice));
    }
    // the sample keeps its pixels; its per-subject counts follow the new tables
    gsvr_status s2 = finish_sample(ctx);
    if (s2) return s2;
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status gsvr_get_subject_losses(gsvr_ctx *ctx, double *out, int32_t n) {
    if (check_ctx(ctx) || !out || n < ctx->n_subj) return GSVR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(out, ctx->d_subj_loss.p, sizeof(double) * ctx->n_subj, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GSVR_OK;
}

// ---------------------------------------------- normalised top-K form (F1)
int topk_cap_px(gsvr_ctx *ctx) { return std::max(ctx->n_mask, 1); }

gsvr_status topk_ensure(gsvr_ctx *ctx) {
    const size_t N = (size_t)std::max<int64_t>(ctx->N, 1), cap = (size_t)topk_cap_px(ctx);
    const size_t nb = (cap + 63) / 64;  // forward blocks of 64 or 128 threads
    const bool need = ctx->d_topk_keys.n < N || ctx->d_topk_gacc.n < 10 * N ||
                      ctx->d_topk_nbr.n < cap * (size_t)ctx->topk_K || ctx->d_topk_loss_part.n < nb ||
                      ctx->d_topk_hist.n < sort_hist_size((int)N) ||
                      ctx->d_scan_bsum.n < scan_scratch_blocks(ctx) + 1 || ctx->topk_n_dev != ctx->N;
    if (!need) return GSVR_OK;
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "top-K buffers must be sized before graph capture");
    CK(ctx->d_topk_grid.ensure(1));
    CK(ctx->d_topk_keys.ensure(N));
    CK(ctx->d_topk_keys_sorted.ensure(N));
    CK(ctx->d_topk_gidx.ensure(N));
    CK(ctx->d_topk_gm.ensure(N));
    CK(ctx->d_topk_kalt.ensure(N));
    CK(ctx->d_topk_valt.ensure(N));
    CK(ctx->d_topk_hist.ensure(sort_hist_size((int)N)));
    CK(ctx->d_topk_cstart.ensure(kTopkMaxCells));
    CK(ctx->d_topk_cend.ensure(kTopkMaxCells));
    CK(ctx->d_topk_nbr.ensure(cap * (size_t)ctx->topk_K));
    CK(ctx->d_topk_ncnt.ensure(cap));
    CK(ctx->d_topk_pstat.ensure(cap));
    CK(ctx->d_topk_loss_part.ensure(nb));
    CK(ctx->d_topk_gacc.ensure(10 * N));
    CK(ctx->d_topk_n.ensure(1));
    CK(ensure_scan_scratch(ctx));
    const int n = (int)ctx->N;
    CK(cudaMemcpyAsync(ctx->d_topk_n.p, &n, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->topk_n_dev = ctx->N;
    ctx->topk_calls = 0;  // a new Gaussian count: the next forward rebuilds the grid
    return GSVR_OK;
}

TopkArgs topk_args(gsvr_ctx *ctx) {
    TopkArgs a{};
    a.theta = ctx->d_theta.p;
    a.gpre = ctx->d_gpre.p;
    a.slices = ctx->d_slices.p;
    a.N = (int)ctx->N;
    a.M = ctx->M;
    a.sampled = ctx->d_sampled.p;
    a.n_sampled = &ctx->d_counters.p->n_sampled;
    a.I_obs = ctx->d_I.p;
    a.pred = ctx->d_pred.p;
    a.rbar = ctx->d_rbar.p;
    a.pstat = ctx->d_topk_pstat.p;
    a.nbr = ctx->d_topk_nbr.p;
    a.ncnt = ctx->d_topk_ncnt.p;
    a.loss_part = ctx->d_topk_loss_part.p;
    a.grid = ctx->d_topk_grid.p;
    a.cell_start = ctx->d_topk_cstart.p;
    a.cell_end = ctx->d_topk_cend.p;
    a.gidx = ctx->d_topk_gidx.p;
    a.gm = ctx->d_topk_gm.p;
    a.gacc = ctx->d_topk_gacc.p;
    a.pose_acc = ctx->d_pose_acc.p;
    a.K = ctx->topk_K;
    a.delta = ctx->topk_delta;
    a.cap_px = topk_cap_px(ctx);
    a.l1 = ctx->loss_kind;
    a.slw = ctx->slw_on ? ctx->d_slw.p : nullptr;
    a.slw_gacc = ctx->d_slw_gacc.p;
    a.status = ctx->d_status.p;
    a.n_weight = ctx->sample_total;
    return a;
}

gsvr_status topk_forward(gsvr_ctx *ctx) {
    if (ctx->n_subj > 1) return fail(ctx, GSVR_ERR_STATE, "the top-K form takes one subject");
    if (gsvr_status s = topk_ensure(ctx)) return s;
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->N;
    stage_begin(ctx, GSVR_STAGE_BIN);
    if (ctx->topk_calls % ctx->topk_refresh == 0) {
        launch_topk_grid(ctx->d_theta.p, N, ctx->topk_per_cell, ctx->d_topk_grid.p, ctx->d_topk_keys.p, st);
        SortScratch ss{ctx->d_topk_kalt.p, ctx->d_topk_valt.p, ctx->d_topk_hist.p, scan_scratch(ctx)};
        CK(radix_sort_pairs(ctx->d_topk_keys.p, nullptr, ctx->d_topk_keys_sorted.p, ctx->d_topk_gidx.p,
                            ctx->d_topk_n.p, N, 16, ss, st));
        CK(cudaMemsetAsync(ctx->d_topk_cstart.p, 0, sizeof(int) * kTopkMaxCells, st));
        CK(cudaMemsetAsync(ctx->d_topk_cend.p, 0, sizeof(int) * kTopkMaxCells, st));
        launch_topk_cell_ranges(ctx->d_topk_keys_sorted.p, N, ctx->d_topk_cstart.p, ctx->d_topk_cend.p, st);
        launch_topk_gather_means(ctx->d_theta.p, ctx->d_topk_gidx.p, N, ctx->d_topk_gm.p, st);
    }
    stage_end(ctx, GSVR_STAGE_BIN);
    stage_begin(ctx, GSVR_STAGE_FWD_EVAL);
    launch_topk_forward(topk_args(ctx), topk_cap_px(ctx), ctx->d_loss.p, st);
    if (ctx->lambda_reg > 0.f) launch_scale_reg_loss(ctx->d_theta.p, N, ctx->lambda_reg, ctx->s_target, ctx->d_loss.p, st);
    if (ctx->slw_on) launch_slw_grad(ctx->d_slw_gacc.p, 2 * ctx->M, ctx->d_slw_grad.p, st);
    stage_end(ctx, GSVR_STAGE_FWD_EVAL);
    CK(cudaGetLastError());
    ++ctx->topk_calls;
    ctx->fwd_valid = true;
    return GSVR_OK;
}

gsvr_status topk_backward(gsvr_ctx *ctx) {
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->N, M = ctx->M;
    stage_begin(ctx, GSVR_STAGE_BWD_EVAL);
    CK(cudaMemsetAsync(ctx->d_topk_gacc.p, 0, sizeof(float) * 10 * (size_t)N, st));
    CK(cudaMemsetAsync(ctx->d_pose_acc.p, 0, sizeof(double) * 12 * M, st));
    launch_topk_backward(topk_args(ctx), topk_cap_px(ctx), st);
    stage_end(ctx, GSVR_STAGE_BWD_EVAL);
    stage_begin(ctx, GSVR_STAGE_GRAD);
    launch_topk_epilogue(ctx->d_theta.p, ctx->d_topk_gacc.p, N, ctx->d_grad.p, st);
    if (ctx->lambda_reg > 0.f) launch_scale_reg_grad(ctx->d_theta.p, N, ctx->lambda_reg, ctx->s_target, ctx->d_grad.p, st);
    launch_pose_grad(ctx->d_pose_acc.p, ctx->d_static.p, ctx->d_theta.p + 11LL * N, ctx->d_grad.p + 11LL * N, M, st);
    stage_end(ctx, GSVR_STAGE_GRAD);
    CK(cudaGetLastError());
    return GSVR_OK;
}

gsvr_status gsvr_forward(gsvr_ctx *ctx) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss || !ctx->have_obs || !ctx->have_sample)
        return fail(ctx, GSVR_ERR_STATE, "set stacks, observations and Gaussians before gsvr_forward");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->N, M = ctx->M;
    Counters *cnt = ctx->d_counters.p;
    const bool grow = !ctx->cfg.fixed_capacity;
    if (ctx->slw_on && ctx->d_slw_tile.n < 2 * (size_t)std::max(ctx->n_tiles, 1)) {
        if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "per-tile slice-weight buffer must exist before capture");
        CK(ctx->d_slw_tile.ensure(2 * (size_t)std::max(ctx->n_tiles, 1)));
    }
    stage_begin(ctx, GSVR_STAGE_PREP);
    CK(cudaMemsetAsync(&cnt->pairs, 0, sizeof(unsigned long long), st));
    if (ctx->slw_on) CK(cudaMemsetAsync(ctx->d_slw_gacc.p, 0, sizeof(double) * 2 * (size_t)M, st));
    launch_gauss_prep(ctx->d_theta.p, N, ctx->d_gpre.p, ctx->d_status.p, st);
    launch_pose_prep(ctx->d_theta.p + 11LL * N, ctx->d_static.p, ctx->d_slices.p, M, ctx->d_status.p, st);
    stage_end(ctx, GSVR_STAGE_PREP);
    if (ctx->topk_K > 0) return topk_forward(ctx);
    stage_begin(ctx, GSVR_STAGE_BIN);

    BinArgs b{};
    b.theta = ctx->d_theta.p;
    b.gpre = ctx->d_gpre.p;
    b.slices = ctx->d_slices.p;
    b.N = N;
    b.M = M;
    b.rc2 = ctx->rc2;
    b.norm_mode = ctx->cfg.norm_mode;
    b.tile_w = ctx->tile_w;
    b.tile_h = ctx->tile_h;
    b.qcut = (float)std::log2((double)ctx->cfg.cutoff_rel);
    b.gauss_subject = ctx->multi_gauss ? ctx->d_gauss_subject.p : nullptr;
    b.subj_active = ctx->multi_gauss && !ctx->h_subj_active.empty() ? ctx->d_subj_active.p : nullptr;
    b.subj_slice_first = ctx->d_subj_slice_first.p;
    b.tile_px_start = ctx->d_tile_px_start.p;
    b.tile_px_end = ctx->d_tile_px_end.p;
    b.rec_cnt = ctx->d_rec_cnt.p;
    b.status = ctx->d_status.p;
    {  // candidate masks (single-subject contexts): the emit pass replays the count pass's tests
        const size_t words = (size_t)((M + 31) / 32) * (size_t)std::max(N, 1);
        if (!ctx->multi_gauss && ctx->d_cand_mask.n < words) {
            if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "candidate masks must exist before capture");
            CK(ctx->d_cand_mask.ensure(words));
        }
        b.cand_mask = ctx->multi_gauss ? nullptr : ctx->d_cand_mask.p;
    }
    launch_cand_count(b, st);
    CK(cudaGetLastError());
    CK(scan_exclusive(ctx->d_rec_cnt.p, ctx->d_rec_off.p, nullptr, N, N, &cnt->n_rec, scan_scratch(ctx), st));
    int n_rec_max = ctx->cap_rec;
    if (grow) {
        int n_rec = 0;
        CK(cudaMemcpyAsync(&n_rec, &cnt->n_rec, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (n_rec > ctx->cap_rec) {
            gsvr_status s = ensure_rec_capacity(ctx, (int64_t)n_rec + n_rec / 4 + 1024);
            if (s) return s;
        }
        n_rec_max = n_rec;
        ctx->last_n_rec = n_rec;
    }
    b.rec_off = ctx->d_rec_off.p;
    b.n_rec = &cnt->n_rec;
    b.cand = ctx->d_cand.p;
    b.rec = ctx->d_rec.p;
    b.rec_tiles = ctx->d_rec_tiles.p;
    b.rec_nkeys = ctx->d_rec_nkeys.p;
    b.rec_mask = ctx->d_rec_mask.p;
    b.cap_rec = ctx->cap_rec;
    launch_cand_emit(b, st);
    launch_records(b, n_rec_max, st);
    CK(cudaGetLastError());
    CK(scan_exclusive(ctx->d_rec_nkeys.p, ctx->d_key_off.p, &cnt->n_rec, 0, std::max(n_rec_max, 0), &cnt->n_keys,
                      scan_scratch(ctx), st));
    int n_keys_max = ctx->cap_keys;
    if (grow) {
        int n_keys = 0;
        CK(cudaMemcpyAsync(&n_keys, &cnt->n_keys, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (n_keys > ctx->cap_keys) {
            gsvr_status s = ensure_key_capacity(ctx, (int64_t)n_keys + n_keys / 4 + 4096);
            if (s) return s;
        }
        n_keys_max = n_keys;
        ctx->last_n_keys = n_keys;
    }
    KeyArgs k{};
    k.rec = ctx->d_rec.p;
    k.cand = ctx->d_cand.p;
    k.rec_tiles = ctx->d_rec_tiles.p;
    k.rec_nkeys = ctx->d_rec_nkeys.p;
    k.rec_mask = ctx->d_rec_mask.p;
    k.mom = ctx->d_mom.p;
    k.key_off = ctx->d_key_off.p;
    k.slices = ctx->d_slices.p;
    k.tile_px_start = ctx->d_tile_px_start.p;
    k.tile_px_end = ctx->d_tile_px_end.p;
    k.n_rec = &cnt->n_rec;
    k.cap_rec = ctx->cap_rec;
    k.cap_keys = ctx->cap_keys;
    k.tile_w = ctx->tile_w;
    k.tile_h = ctx->tile_h;
    k.n_tiles = ctx->n_tiles;
    k.qcut = b.qcut;
    k.keys = ctx->d_keys.p;
    k.key_rec = ctx->d_key_rec.p;
    k.status = ctx->d_status.p;
    launch_key_emit(k, n_rec_max, st);
    CK(cudaGetLastError());
    TileSortScratch ss{ctx->d_keys_alt.p, ctx->d_vals_alt.p, ctx->d_hist.p, scan_scratch(ctx)};
    if (n_keys_max > 0)
        CK(sort_tile_keys(ctx->d_keys.p, ctx->d_key_rec.p, ctx->d_keys_sorted.p, ctx->d_tref.p, &cnt->n_keys,
                          n_keys_max, ctx->sort_bits, ss, ctx->d_status.p, st));
    launch_tile_rec_ranges(ctx->d_keys_sorted.p, &cnt->n_keys, n_keys_max, ctx->n_tiles, ctx->d_tile_rec_start.p,
                           ctx->d_tile_rec_end.p, st);
    {
        gsvr_status si = ensure_item_capacity(ctx);
        if (si) return si;
    }
    launch_items(ctx->d_tile_px_start.p, ctx->d_tile_px_end.p, ctx->d_tile_rec_start.p, ctx->d_tile_rec_end.p,
                 ctx->n_tiles, ctx->d_item_cnt.p, nullptr, nullptr, 0, 0, st, &cnt->pairs, ctx->d_pairs_total.p);
    CK(scan_exclusive(ctx->d_item_cnt.p, ctx->d_item_first.p, nullptr, ctx->n_tiles, ctx->n_tiles, &cnt->n_items,
                      scan_scratch(ctx), st));
    launch_items(nullptr, nullptr, nullptr, nullptr, ctx->n_tiles, nullptr, ctx->d_item_first.p, ctx->d_item_tile.p,
                 ctx->cap_items, 1, st);
    if (ctx->queue_order) {
        SortScratch is{ctx->d_item_key_alt.p, ctx->d_item_val_alt.p, ctx->d_item_hist.p, scan_scratch(ctx)};
        launch_item_order(ctx->d_item_tile.p, ctx->d_item_first.p, ctx->d_tile_rec_start.p, ctx->d_tile_rec_end.p,
                          &cnt->n_items, ctx->cap_items, ctx->d_item_key.p, ctx->d_item_key_sorted.p,
                          ctx->d_item_order.p, is, st);
    }
    stage_end(ctx, GSVR_STAGE_BIN);
    ctx->grid_items = ctx->n_tiles + n_keys_max / kItemRecs + 2;
    EvalArgs e = eval_args(ctx, ctx->grid_items);
    if (ctx->test_wait_forwards > 0) {
        e.wait_test_ns = ctx->test_wait_ns;
        --ctx->test_wait_forwards;
    }
    stage_begin(ctx, GSVR_STAGE_FWD_EVAL);
    launch_forward(e, st);
    stage_end(ctx, GSVR_STAGE_FWD_EVAL);
    if (ctx->slw_on) launch_slw_slices(ctx->d_slw_tile.p, ctx->d_slices.p, M, ctx->d_slw_gacc.p, st);
    launch_loss_reduce(ctx->d_tile_loss.p, ctx->n_tiles, ctx->d_subj_tile_first.p, ctx->n_subj, ctx->d_subj_loss.p,
                       ctx->d_loss.p, ctx->d_status.p, st);
    if (ctx->lambda_reg > 0.f) launch_scale_reg_loss(ctx->d_theta.p, N, ctx->lambda_reg, ctx->s_target, ctx->d_loss.p, st);
    if (ctx->slw_on) launch_slw_grad(ctx->d_slw_gacc.p, 2 * M, ctx->d_slw_grad.p, st);
    CK(cudaGetLastError());
    ctx->fwd_valid = true;
    return GSVR_OK;
}

gsvr_status gsvr_backward(gsvr_ctx *ctx) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->fwd_valid) return fail(ctx, GSVR_ERR_STATE, "gsvr_backward needs a current gsvr_forward");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->N, M = ctx->M;
    if (ctx->topk_K > 0) return topk_backward(ctx);
    EvalArgs e = eval_args(ctx, ctx->grid_items);
    stage_begin(ctx, GSVR_STAGE_BWD_EVAL);
    launch_backward(e, (int)ctx->n_mask, st);
    stage_end(ctx, GSVR_STAGE_BWD_EVAL);
    stage_begin(ctx, GSVR_STAGE_GRAD);
    CK(cudaMemsetAsync(ctx->d_pose_acc.p, 0, sizeof(double) * 12 * M, st));
    GradArgs a{};
    a.theta = ctx->d_theta.p;
    a.gpre = ctx->d_gpre.p;
    a.slices = ctx->d_slices.p;
    a.rec = ctx->d_rec.p;
    a.rec_off = ctx->d_rec_off.p;
    a.cand = ctx->d_cand.p;
    a.key_off = ctx->d_key_off.p;
    a.mom = ctx->d_mom.p;
    a.keys = ctx->d_keys.p;
    a.n_tiles = ctx->n_tiles;
    a.N = N;
    a.M = M;
    a.rc2 = ctx->rc2;
    a.norm_mode = ctx->cfg.norm_mode;
    a.grad = ctx->d_grad.p;
    a.pose_acc = ctx->d_pose_acc.p;
    a.gauss_subject = ctx->multi_gauss ? ctx->d_gauss_subject.p : nullptr;
    a.subj_slice_first = ctx->d_subj_slice_first.p;
    a.smem_slices = 1536;  // at most 72 KB of shared float accumulators per block
    a.h_gauss_first = ctx->h_subj_gauss_first.data();
    a.h_slice_first = ctx->h_subj_slice_first.data();
    a.n_subj = ctx->n_subj;
    a.cap_rec = ctx->cap_rec;
    a.cap_keys = ctx->cap_keys;
    launch_gauss_grad(a, st);
    if (ctx->lambda_reg > 0.f) launch_scale_reg_grad(ctx->d_theta.p, N, ctx->lambda_reg, ctx->s_target, ctx->d_grad.p, st);
    launch_pose_grad(ctx->d_pose_acc.p, ctx->d_static.p, ctx->d_theta.p + 11LL * N, ctx->d_grad.p + 11LL * N, M, st);
    stage_end(ctx, GSVR_STAGE_GRAD);
    CK(cudaGetLastError());
    return GSVR_OK;
}

gsvr_status adam_launch(gsvr_ctx *ctx, const gsvr_adam_cfg *cfg, int64_t step, const unsigned long long *d_step) {
    const float b1 = cfg->beta1 == 0.f ? 0.9f : cfg->beta1;
    const float b2 = cfg->beta2 == 0.f ? 0.999f : cfg->beta2;
    const float eps = cfg->eps == 0.f ? 1e-8f : cfg->eps;
    const float gamma = cfg->gamma == 0.f ? 1.0f : cfg->gamma;
    if (!(b1 > 0.f && b1 < 1.f && b2 > 0.f && b2 < 1.f && eps > 0.f && gamma > 0.f) || cfg->step_every < 0)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad Adam betas, eps or schedule");
    const float lr[6] = {cfg->lr_mu, cfg->lr_ls, cfg->lr_q, cfg->lr_c, cfg->lr_rot, cfg->lr_trans};
    stage_begin(ctx, GSVR_STAGE_ADAM);
    launch_adam(ctx->d_theta.p, ctx->d_grad.p, ctx->d_m.p, ctx->d_v.p, (int)ctx->N, ctx->M, lr, b1, b2, eps,
                cfg->step_every, gamma, step, d_step, ctx->d_counters.p->adam_scal,
                ctx->any_frozen ? ctx->d_frozen.p : nullptr, ctx->stream);
    if (ctx->slw_on)
        launch_adam_slw(ctx->d_slw.p, ctx->d_slw_grad.p, ctx->d_slw_m.p, ctx->d_slw_v.p, ctx->M, ctx->lr_slw_sig,
                        ctx->lr_slw_omg, b1, b2, eps, cfg->step_every, gamma, step, d_step,
                        ctx->d_counters.p->adam_scal, ctx->any_frozen ? ctx->d_frozen.p : nullptr, ctx->stream);
    stage_end(ctx, GSVR_STAGE_ADAM);
    CK(cudaGetLastError());
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status gsvr_adam_step(gsvr_ctx *ctx, const gsvr_adam_cfg *cfg, int64_t step) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_gaussians first");
    if (!cfg || step < 1) return fail(ctx, GSVR_ERR_INVALID_ARG, "adam config NULL or step < 1");
    DeviceGuard g(ctx->device);
    return adam_launch(ctx, cfg, step, nullptr);
}

gsvr_status gsvr_set_sample_total(gsvr_ctx *ctx, int64_t n_total) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (n_total < 0 || n_total > (int64_t)1 << 40) return fail(ctx, GSVR_ERR_INVALID_ARG, "n_total must be in [0, 2^40]");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_sample_total during graph capture");
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    ctx->sample_total = n_total;
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status gsvr_test_wait_timeout(gsvr_ctx *ctx, int32_t n_forwards, int64_t limit_ns) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (n_forwards < 0 || limit_ns < 1000 || limit_ns > 1000000000)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "n_forwards >= 0 and limit_ns in [1e3, 1e9] needed");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_test_wait_timeout during graph capture");
    ctx->test_wait_forwards = n_forwards;
    ctx->test_wait_ns = limit_ns;
    return GSVR_OK;
}

gsvr_status gsvr_set_step(gsvr_ctx *ctx, int64_t step) {
    if (check_ctx(ctx) || step < 0) return GSVR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const unsigned long long v = (unsigned long long)step;
    CK(cudaMemcpyAsync(&ctx->d_counters.p->step, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GSVR_OK;
}

gsvr_status gsvr_graph_capture(gsvr_ctx *ctx, int64_t n_per_subject, const gsvr_adam_cfg *cfg) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->cfg.fixed_capacity) return fail(ctx, GSVR_ERR_STATE, "graph capture needs fixed_capacity = 1");
    if (!ctx->have_gauss || !ctx->have_obs || !ctx->have_sample || !cfg)
        return fail(ctx, GSVR_ERR_STATE, "set stacks, observations, Gaussians and a sample before capturing");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    if (!st) return fail(ctx, GSVR_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    CK(cudaStreamSynchronize(st));
    {
        gsvr_status si = ensure_item_capacity(ctx);
        if (si) return si;
    }
    if (ctx->topk_K > 0) {
        if (gsvr_status sk = topk_ensure(ctx)) return sk;
    }
    int64_t n_out = -1;
    if (n_per_subject >= 0) {
        n_out = subject_out_first(ctx, n_per_subject);
        if (n_out < 0) return fail(ctx, GSVR_ERR_CUDA, "upload of the sample offsets failed");
    }
    if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    if (ctx->graph) {
        cudaGraphDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    gsvr_status s = GSVR_OK;
    const unsigned long long *dstep = &ctx->d_counters.p->step;
    if (n_out >= 0)
        s = sample_ranges(ctx, ctx->n_subj, ctx->d_subj_mask_first.p, ctx->d_subj_out_first.p, (int)n_out, 0, dstep);
    if (!s) s = gsvr_forward(ctx);
    if (!s) s = gsvr_backward(ctx);
    if (!s) s = adam_launch(ctx, cfg, 1, dstep);
    if (!s) launch_advance_step(&ctx->d_counters.p->step, st);
    ctx->capturing = false;
    cudaGraph_t gph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &gph);
    if (s) {
        if (gph) cudaGraphDestroy(gph);
        cudaGetLastError();
        return s;
    }
    if (ec != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GSVR_ERR_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(ec));
    }
    ctx->graph = gph;
    CK(cudaGraphInstantiate(&ctx->graph_exec, gph, 0));
    return GSVR_OK;
}

gsvr_status gsvr_graph_launch(gsvr_ctx *ctx, int32_t iterations) {
    if (check_ctx(ctx) || iterations < 0) return GSVR_ERR_INVALID_ARG;
    if (!ctx->graph_exec) return fail(ctx, GSVR_ERR_STATE, "no captured graph");
    DeviceGuard g(ctx->device);
    for (int k = 0; k < iterations; ++k) CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    note_launches(0);
    ctx->fwd_valid = false;
    return GSVR_OK;
}

gsvr_status gsvr_sync_status(gsvr_ctx *ctx) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    unsigned s = 0;
    CK(cudaMemcpyAsync(&s, ctx->d_status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (s) CK(cudaMemsetAsync(ctx->d_status.p, 0, sizeof(unsigned), ctx->stream));
    if (s & ST_CAPACITY) return fail(ctx, GSVR_ERR_CAPACITY, "record or key capacity exceeded");
    if (s & ST_NONFINITE) return fail(ctx, GSVR_ERR_NONFINITE, "non-finite parameter, pose or loss");
    if (s & ST_TIMEOUT) return fail(ctx, GSVR_ERR_TIMEOUT, "a bounded device wait ran out");
    if (s & ST_INDEX) return fail(ctx, GSVR_ERR_INVALID_ARG, "pixel index out of range in a sample list");
    if (s & ST_SHAPE) return fail(ctx, GSVR_ERR_INVALID_ARG, "forward launch shape exceeds the kernel's shared buffers");
    return GSVR_OK;
}

gsvr_status gsvr_step_host(gsvr_ctx *ctx, const float *theta, const int32_t *idx, int64_t n, float *grad_out,
                           double *loss_out) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss || !ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "context not initialised");
    if (!theta) return fail(ctx, GSVR_ERR_INVALID_ARG, "theta is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const size_t np = (size_t)(11 * ctx->N + 6 * ctx->M);
    CK(cudaMemcpyAsync(ctx->d_theta.p, theta, sizeof(float) * np, cudaMemcpyHostToDevice, st));
    gsvr_status s = gsvr_set_pixel_sample(ctx, idx, n, GSVR_MEM_HOST);
    if (s) return s;
    s = gsvr_forward(ctx);
    if (s) return s;
    s = gsvr_backward(ctx);
    if (s) return s;
    if (grad_out) CK(cudaMemcpyAsync(grad_out, ctx->d_grad.p, sizeof(float) * np, cudaMemcpyDeviceToHost, st));
    if (loss_out) CK(cudaMemcpyAsync(loss_out, ctx->d_loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    return gsvr_sync_status(ctx);
}

gsvr_status gsvr_timing_reset(gsvr_ctx *ctx) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    fold_marks(ctx);
    for (int k = 0; k < GSVR_N_STAGES; ++k) {
        ctx->ms[k] = 0.0;
        ctx->calls[k] = 0;
    }
    CK(cudaMemset(ctx->d_pairs_total.p, 0, sizeof(unsigned long long)));
    CK(cudaMemset(ctx->d_bwd_pairs_total.p, 0, sizeof(unsigned long long)));
    ctx->launches_at_reset = launch_count();
    return GSVR_OK;
}

gsvr_status gsvr_get_kernel_times(gsvr_ctx *ctx, gsvr_kernel_times *out) {
    if (check_ctx(ctx) || !out) return GSVR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    fold_marks(ctx);
    unsigned long long pt = 0, pb = 0;
    CK(cudaMemcpy(&pt, ctx->d_pairs_total.p, sizeof(pt), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&pb, ctx->d_bwd_pairs_total.p, sizeof(pb), cudaMemcpyDeviceToHost));
    for (int k = 0; k < GSVR_N_STAGES; ++k) {
        out->ms[k] = ctx->ms[k];
        out->calls[k] = ctx->calls[k];
    }
    out->pairs_evaluated = (int64_t)pt;
    out->bwd_pairs_evaluated = (int64_t)pb;
    out->kernel_launches = launch_count() - ctx->launches_at_reset;
    return GSVR_OK;
}

gsvr_status gsvr_count_pairs(gsvr_ctx *ctx, int64_t *useful, int64_t *evaluated) {
    if (check_ctx(ctx) || !useful || !evaluated) return GSVR_ERR_INVALID_ARG;
    if (!ctx->fwd_valid) return fail(ctx, GSVR_ERR_STATE, "gsvr_count_pairs needs a current gsvr_forward");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    Counters *cnt = ctx->d_counters.p;
    CK(cudaMemsetAsync(ctx->d_useful.p, 0, sizeof(unsigned long long), st));
    EvalArgs e = eval_args(ctx, ctx->grid_items);
    e.useful = ctx->d_useful.p;
    e.qcut = (float)std::log2((double)ctx->cfg.cutoff_rel);
    launch_count_pairs(e, st);
    CK(cudaGetLastError());
    unsigned long long u = 0;
    Counters c{};
    CK(cudaMemcpyAsync(&u, ctx->d_useful.p, sizeof(u), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&c, cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *useful = (int64_t)u;
    *evaluated = (int64_t)c.pairs;
    return GSVR_OK;
}

gsvr_status gsvr_get_sample(gsvr_ctx *ctx, int32_t *out, int64_t cap, int64_t *n_out) {
    if (check_ctx(ctx) || !n_out || cap < 0 || (cap > 0 && !out)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_sample) return fail(ctx, GSVR_ERR_STATE, "no sample");
    DeviceGuard g(ctx->device);
    Counters c{};
    CK(cudaMemcpyAsync(&c, ctx->d_counters.p, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *n_out = c.n_sampled;
    const int64_t n = std::min<int64_t>(cap, c.n_sampled);
    if (n > 0) CK(cudaMemcpy(out, ctx->d_sampled.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
    return GSVR_OK;
}

gsvr_status gsvr_get_views(gsvr_ctx *ctx, gsvr_views *out) {
    if (check_ctx(ctx) || !out) return GSVR_ERR_INVALID_ARG;
    out->theta = ctx->d_theta.p;
    out->grad = ctx->d_grad.p;
    out->adam_m = ctx->d_m.p;
    out->adam_v = ctx->d_v.p;
    out->pred = ctx->d_pred.p;
    out->rbar = ctx->d_rbar.p;
    out->loss = ctx->d_loss.p;
    out->n_gauss = ctx->N;
    out->n_slices = ctx->M;
    out->n_pixels = ctx->P;
    out->n_params = 11 * ctx->N + 6 * ctx->M;
    return GSVR_OK;
}

gsvr_status gsvr_get_stats(gsvr_ctx *ctx, gsvr_stats *out) {
    if (check_ctx(ctx) || !out) return GSVR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    Counters c{};
    CK(cudaMemcpyAsync(&c, ctx->d_counters.p, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out->n_sampled = c.n_sampled;
    out->n_records = c.n_rec;
    out->n_keys = c.n_keys;
    out->pairs_evaluated = (int64_t)c.pairs;
    out->n_tiles = ctx->n_tiles;
    out->tile_px_max = (int64_t)ctx->tile_w * ctx->tile_h;
    out->cap_records = ctx->cap_rec;
    out->cap_keys = ctx->cap_keys;
    return GSVR_OK;
}

}  // extern "C"

// ------------------------------------------------------------- launch shape
namespace {
gsvr_status check_tiling(gsvr_ctx *ctx, const gsvr_tiling &t) {
    const int th = t.tile_h ? t.tile_h : 16, tw = t.tile_w ? t.tile_w : 16;
    if (th < 4 || th > 32 || tw < 4 || tw > 32)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "tile sides must lie in [4, 32]");
    if (t.fwd_px_per_thread != 0 && t.fwd_px_per_thread != 1 && t.fwd_px_per_thread != 2 &&
        t.fwd_px_per_thread != 4 && t.fwd_px_per_thread != 8 && t.fwd_px_per_thread != 16)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "fwd_px_per_thread must be 0, 1, 2, 4, 8 or 16");
    const int pxr = fwd_pxr(tw, t.fwd_px_per_thread);
    if (th * ((tw + pxr - 1) / pxr) > 256)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "tile_h * ceil(tile_w / px_per_thread) must be <= 256");
    if (!fwd_shape_fits(tw, th, pxr))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "forward groups x tile pixels exceed the kernel's shared buffer");
    if (t.fwd_blocks_per_sm < -1 || t.fwd_blocks_per_sm > 64 || t.bwd_blocks_per_sm < -1 || t.bwd_blocks_per_sm > 64)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "blocks per SM must lie in [-1, 64]");
    if (t.queue_order != 0 && t.queue_order != 1) return fail(ctx, GSVR_ERR_INVALID_ARG, "queue_order must be 0 or 1");
    return GSVR_OK;
}

void drop_graph(gsvr_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
}

gsvr_status tune_iteration(gsvr_ctx *ctx, int64_t n_per_subject, int step) {
    gsvr_status s = GSVR_OK;
    if (n_per_subject > 0)
        s = ctx->n_subj > 1 ? gsvr_sample_pixels_subjects(ctx, n_per_subject, (uint64_t)step)
                            : gsvr_sample_pixels(ctx, std::min<int64_t>(n_per_subject, ctx->n_mask), (uint64_t)step);
    if (!s) s = gsvr_forward(ctx);
    if (!s) s = gsvr_backward(ctx);
    return s;
}
}  // namespace

extern "C" {

gsvr_status gsvr_get_tiling(gsvr_ctx *ctx, gsvr_tiling *out) {
    if (check_ctx(ctx) || !out) return GSVR_ERR_INVALID_ARG;
    out->tile_h = ctx->tile_h;
    out->tile_w = ctx->tile_w;
    out->fwd_px_per_thread = ctx->fwd_pxr_req;
    out->fwd_blocks_per_sm = ctx->fwd_bps;
    out->bwd_blocks_per_sm = ctx->bwd_bps;
    out->queue_order = ctx->queue_order;
    out->ms = 0.f;
    return GSVR_OK;
}

gsvr_status gsvr_get_topk_neighbors(gsvr_ctx *ctx, int32_t *pix, int32_t *nbr, int32_t *cnt, int64_t cap,
                                    int64_t *n_out) {
    if (check_ctx(ctx) || !n_out) return GSVR_ERR_INVALID_ARG;
    if (ctx->topk_K <= 0 || !ctx->fwd_valid) return fail(ctx, GSVR_ERR_STATE, "needs a top-K forward");
    DeviceGuard g(ctx->device);
    int ns = 0;
    CK(cudaMemcpyAsync(&ns, &ctx->d_counters.p->n_sampled, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ns = std::min(ns, topk_cap_px(ctx));
    *n_out = ns;
    if (!pix && !nbr && !cnt) return GSVR_OK;
    if (cap < ns || !pix || !nbr || !cnt) return fail(ctx, GSVR_ERR_INVALID_ARG, "need pix, nbr, cnt with cap >= n");
    CK(cudaMemcpy(pix, ctx->d_sampled.p, sizeof(int) * (size_t)ns, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nbr, ctx->d_topk_nbr.p, sizeof(int) * (size_t)ns * ctx->topk_K, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt, ctx->d_topk_ncnt.p, sizeof(int) * (size_t)ns, cudaMemcpyDeviceToHost));
    return GSVR_OK;
}

gsvr_status gsvr_init_means(gsvr_ctx *ctx, const float *pose, int64_t n, float lambda_init, uint64_t seed,
                            float *mu, int32_t *pix, int64_t *total_weight) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_stacks || !ctx->have_obs)
        return fail(ctx, GSVR_ERR_STATE, "set stacks and observations before gsvr_init_means");
    if (n < 0 || n > (int64_t)1 << 30 || (n > 0 && !mu) || !(lambda_init >= 0.f && lambda_init <= 1.f))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "need 0 <= n <= 2^30, mu for n > 0, 0 <= lambda_init <= 1");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_init_means during graph capture");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int M = ctx->M;
    const int64_t P = ctx->P;
    std::vector<float> hp((size_t)6 * M, 0.f), th;
    if (pose) {
        if (!finite_all(pose, 6 * M)) return fail(ctx, GSVR_ERR_INVALID_ARG, "non-finite pose");
        std::copy(pose, pose + 6 * M, hp.begin());
    }
    for (const gsvr_stack_desc &d : ctx->h_stack_desc)
        for (int k = 0; k < d.n_slices; ++k) th.push_back(d.thickness);
    CK(ctx->d_init_pose.ensure((size_t)6 * M));
    CK(ctx->d_init_thick.ensure((size_t)M));
    CK(ctx->d_init_w.ensure((size_t)P));
    CK(ctx->d_init_c.ensure((size_t)P));
    CK(ctx->d_init_s.ensure((size_t)(P + 4095) / 4096 + 1));
    CK(cudaMemcpyAsync(ctx->d_init_pose.p, hp.data(), sizeof(float) * hp.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_init_thick.p, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, st));
    // slice frames of these poses (the next forward rebuilds them from the parameters)
    launch_pose_prep(ctx->d_init_pose.p, ctx->d_static.p, ctx->d_slices.p, M, ctx->d_status.p, st);
    launch_init_weights(ctx->d_I.p, ctx->d_mask.p, ctx->d_slices.p, M, P, lambda_init, ctx->d_init_w.p,
                        ctx->d_init_c.p, ctx->d_init_s.p, st);
    int64_t T = 0;
    CK(cudaMemcpyAsync(&T, ctx->d_init_c.p + (P - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->fwd_valid = false;
    if (total_weight) *total_weight = T;
    if (T <= 0) return fail(ctx, GSVR_ERR_INVALID_ARG, "no masked pixel carries weight (flat slices with lambda_init 0)");
    launch_init_draw(ctx->d_init_c.p, P, seed, n, ctx->d_slices.p, M, ctx->d_init_thick.p, mu, pix, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return GSVR_OK;
}

gsvr_status gsvr_set_slice_weights(gsvr_ctx *ctx, int32_t enable, float lr_log_sigma, float lr_log_omega) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!(lr_log_sigma >= 0.f) || !(lr_log_omega >= 0.f) || !std::isfinite(lr_log_sigma) ||
        !std::isfinite(lr_log_omega))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "slice-weight learning rates must be >= 0 and finite");
    if (!ctx->have_stacks) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_stacks before gsvr_set_slice_weights");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_slice_weights during graph capture");
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    ctx->fwd_valid = false;
    ctx->slw_on = enable != 0;
    ctx->lr_slw_sig = lr_log_sigma;
    ctx->lr_slw_omg = lr_log_omega;
    if (!ctx->slw_on) return GSVR_OK;
    const size_t n = 2 * (size_t)ctx->M;
    CK(ctx->d_slw.ensure(n));
    CK(ctx->d_slw_grad.ensure(n));
    CK(ctx->d_slw_m.ensure(n));
    CK(ctx->d_slw_v.ensure(n));
    CK(ctx->d_slw_gacc.ensure(n));
    CK(ctx->d_slw_tile.ensure(2 * (size_t)std::max(ctx->n_tiles, 1)));
    for (DBuf<float> *b : {&ctx->d_slw, &ctx->d_slw_grad, &ctx->d_slw_m, &ctx->d_slw_v})
        CK(cudaMemsetAsync(b->p, 0, sizeof(float) * n, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_slw_gacc.p, 0, sizeof(double) * n, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GSVR_OK;
}

gsvr_status gsvr_slice_weight_views(gsvr_ctx *ctx, float **params, float **grads, int32_t *M) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->slw_on) return fail(ctx, GSVR_ERR_STATE, "slice weights are off");
    if (params) *params = ctx->d_slw.p;
    if (grads) *grads = ctx->d_slw_grad.p;
    if (M) *M = ctx->M;
    return GSVR_OK;
}

gsvr_status gsvr_set_objective(gsvr_ctx *ctx, int32_t loss_kind, float lambda_reg, float s_target) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if ((loss_kind != 0 && loss_kind != 1) || !(lambda_reg >= 0.f) || !std::isfinite(lambda_reg) ||
        !(s_target > 0.f) || !std::isfinite(s_target))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "objective needs loss_kind 0 or 1, lambda_reg >= 0, s_target > 0");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_objective during graph capture");
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    ctx->loss_kind = loss_kind;
    ctx->lambda_reg = lambda_reg;
    ctx->s_target = s_target;
    ctx->fwd_valid = false;
    return GSVR_OK;
}

// ------------------------------------------------------------ densification
}  // extern "C"

namespace {

template <class T>
void swap_buf(DBuf<T> &a, DBuf<T> &b) {
    std::swap(a.p, b.p);
    std::swap(a.n, b.n);
}

// Statistics sized for the current N, zeroed when N changed since they were.
gsvr_status dens_ensure(gsvr_ctx *ctx) {
    if (ctx->dens_n == ctx->N && ctx->d_dens_acc.p && ctx->d_dens_cnt.p) return GSVR_OK;
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "densification statistics must be sized before graph capture");
    const size_t n = (size_t)std::max<int64_t>(ctx->N, 1);
    CK(ctx->d_dens_acc.ensure(n));
    CK(ctx->d_dens_cnt.ensure(1));
    CK(cudaMemsetAsync(ctx->d_dens_acc.p, 0, sizeof(float4) * n, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_dens_cnt.p, 0, sizeof(int), ctx->stream));
    ctx->dens_n = ctx->N;
    return GSVR_OK;
}

}  // namespace

extern "C" {

gsvr_status gsvr_densify_accumulate(gsvr_ctx *ctx) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_gaussians first");
    DeviceGuard g(ctx->device);
    if (gsvr_status s = dens_ensure(ctx)) return s;
    launch_dens_accum(ctx->d_grad.p, (int)ctx->N, ctx->d_dens_acc.p, ctx->d_dens_cnt.p, ctx->stream);
    CK(cudaGetLastError());
    return GSVR_OK;
}

gsvr_status gsvr_densify_stats(gsvr_ctx *ctx, float *acc, int32_t *count, int32_t set) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_gaussians first");
    if ((ctx->N > 0 && !acc) || !count || (set != 0 && set != 1))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad statistics pointer or direction");
    if (set && *count < 0) return fail(ctx, GSVR_ERR_INVALID_ARG, "negative pass count");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_densify_stats during graph capture");
    DeviceGuard g(ctx->device);
    if (gsvr_status s = dens_ensure(ctx)) return s;
    const size_t bytes = sizeof(float4) * (size_t)ctx->N;
    cudaStream_t st = ctx->stream;
    if (set) {
        if (bytes) CK(cudaMemcpyAsync(ctx->d_dens_acc.p, acc, bytes, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_dens_cnt.p, count, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    } else {
        if (bytes) CK(cudaMemcpyAsync(acc, ctx->d_dens_acc.p, bytes, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(count, ctx->d_dens_cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return GSVR_OK;
}

gsvr_status gsvr_densify(gsvr_ctx *ctx, const gsvr_densify_cfg *cfg, int64_t *counts) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!ctx->have_gauss) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_gaussians first");
    if (!cfg || !std::isfinite(cfg->grad_threshold) || !std::isfinite(cfg->log_scale_threshold) ||
        !(cfg->prune_amplitude >= 0.f) || !std::isfinite(cfg->prune_amplitude) || !(cfg->split_factor > 1.f) ||
        !std::isfinite(cfg->split_factor) || !(cfg->clone_offset >= 0.f) || !std::isfinite(cfg->clone_offset) ||
        (cfg->mass_preserving != 0 && cfg->mass_preserving != 1) || cfg->max_gaussians < 0)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "bad densification configuration");
    if (ctx->n_subj > 1) return fail(ctx, GSVR_ERR_STATE, "densification of a batched context is not supported");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_densify during graph capture");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    if (gsvr_status s = dens_ensure(ctx)) return s;
    const int N = (int)ctx->N, M = ctx->M;
    const int64_t cap = cfg->max_gaussians > 0 ? std::min<int64_t>(cfg->max_gaussians, 1LL << 26) : (1LL << 26);
    int h[4] = {0, 0, 0, 0};  // split, cloned, pruned, new count
    if (N > 0) {
        CK(ctx->d_dens_kind.ensure((size_t)N));
        CK(ctx->d_dens_nout.ensure((size_t)N + 1));
        CK(ctx->d_dens_off.ensure((size_t)N + 1));
        CK(ctx->d_dens_misc.ensure(4));
        CK(cudaMemsetAsync(ctx->d_dens_misc.p, 0, sizeof(int) * 4, st));
        launch_dens_decide(ctx->d_theta.p, N, ctx->d_dens_acc.p, ctx->d_dens_cnt.p, cfg->grad_threshold,
                           cfg->log_scale_threshold, cfg->prune_amplitude, ctx->d_dens_kind.p, ctx->d_dens_nout.p,
                           ctx->d_dens_misc.p, st);
        CK(ensure_scan_scratch(ctx));
        CK(scan_exclusive(ctx->d_dens_nout.p, ctx->d_dens_off.p, nullptr, N, N, ctx->d_dens_misc.p + 3,
                          scan_scratch(ctx), st));
        CK(cudaMemcpyAsync(h, ctx->d_dens_misc.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    const int64_t N2 = N > 0 ? h[3] : 0;
    if (N2 > cap) return fail(ctx, GSVR_ERR_CAPACITY, "densification would exceed max_gaussians; nothing changed");
    if (N > 0 && (h[0] || h[1] || h[2])) {
        const size_t np2 = (size_t)(11 * N2 + 6 * M);
        DBuf<float> t2, m2, v2;
        CK(t2.ensure(np2));
        CK(m2.ensure(np2));
        CK(v2.ensure(np2));
        DensParams p{};
        p.split_factor = cfg->split_factor;
        p.log_split_factor = (float)std::log((double)cfg->split_factor);
        p.split_offset = (float)std::sqrt(1.0 - 1.0 / ((double)cfg->split_factor * (double)cfg->split_factor));
        p.clone_offset = cfg->clone_offset;
        p.mass_preserving = cfg->mass_preserving;
        launch_dens_emit(ctx->d_theta.p, ctx->d_m.p, ctx->d_v.p, N, ctx->d_dens_acc.p, ctx->d_dens_kind.p,
                         ctx->d_dens_off.p, (int)N2, p, t2.p, m2.p, v2.p, st);
        if (M > 0) {
            const size_t pb = sizeof(float) * 6 * (size_t)M;
            CK(cudaMemcpyAsync(t2.p + 11 * N2, ctx->d_theta.p + 11 * (int64_t)N, pb, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(m2.p + 11 * N2, ctx->d_m.p + 11 * (int64_t)N, pb, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(v2.p + 11 * N2, ctx->d_v.p + 11 * (int64_t)N, pb, cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaStreamSynchronize(st));  // the old buffers are read until here
        swap_buf(ctx->d_theta, t2);
        swap_buf(ctx->d_m, m2);
        swap_buf(ctx->d_v, v2);
        ctx->d_grad.release();
        CK(ctx->d_grad.ensure(np2));
        CK(cudaMemsetAsync(ctx->d_grad.p, 0, sizeof(float) * np2, st));
        CK(ctx->d_gpre.ensure((size_t)2 * N2));
        CK(ctx->d_rec_cnt.ensure((size_t)N2 + 1));
        CK(ctx->d_rec_off.ensure((size_t)N2 + 1));
        ctx->N = N2;
        if (gsvr_status s = gauss_capacities(ctx, N2)) return s;
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->graph) cudaGraphDestroy(ctx->graph);
        ctx->graph_exec = nullptr;
        ctx->graph = nullptr;
        ctx->fwd_valid = false;
    }
    ctx->dens_n = -1;  // the statistics restart (sized for the new count)
    if (gsvr_status s = dens_ensure(ctx)) return s;
    CK(cudaStreamSynchronize(st));
    if (counts) {
        counts[0] = ctx->N;
        counts[1] = h[0];
        counts[2] = h[1];
        counts[3] = h[2];
    }
    return GSVR_OK;
}

gsvr_status gsvr_set_topk(gsvr_ctx *ctx, int32_t K, float delta, int32_t refresh_every) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (K < 0 || K > kTopkMaxK || !(delta > 0.f) || !std::isfinite(delta) || refresh_every < 1)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "top-K needs 0 <= K <= 128, delta > 0 finite, refresh_every >= 1");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_topk during graph capture");
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    ctx->topk_K = K;
    ctx->topk_delta = delta;
    ctx->topk_refresh = refresh_every;
    ctx->topk_calls = 0;
    ctx->fwd_valid = false;
    if (K > 0 && ctx->have_gauss) return topk_ensure(ctx);
    return GSVR_OK;
}

gsvr_status gsvr_set_tiling(gsvr_ctx *ctx, const gsvr_tiling *t) {
    if (check_ctx(ctx) || !t) return GSVR_ERR_INVALID_ARG;
    if (gsvr_status s = check_tiling(ctx, *t)) return s;
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_set_tiling during graph capture");
    DeviceGuard g(ctx->device);
    const int th = t->tile_h ? t->tile_h : 16, tw = t->tile_w ? t->tile_w : 16;
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    ctx->fwd_pxr_req = t->fwd_px_per_thread;
    ctx->fwd_bps = t->fwd_blocks_per_sm;
    ctx->bwd_bps = t->bwd_blocks_per_sm;
    ctx->queue_order = t->queue_order;
    ctx->fwd_valid = false;
    if (th == ctx->tile_h && tw == ctx->tile_w) return ctx->have_gauss ? ensure_item_capacity(ctx) : GSVR_OK;
    ctx->tile_h = th;
    ctx->tile_w = tw;
    if (!ctx->have_stacks) return GSVR_OK;
    // Everything in tile order is rebuilt: the stacks, then the observations and
    // mask (kept on the device), the subjects and the frozen slices.
    const std::vector<gsvr_stack_desc> desc = ctx->h_stack_desc;
    const bool had_obs = ctx->have_obs;
    const int n_subj = ctx->n_subj, M = ctx->M;
    const std::vector<int> stack_subject = ctx->h_stack_subject;
    std::vector<int64_t> gauss_count;
    for (int k = 0; k < n_subj && k + 1 < (int)ctx->h_subj_gauss_first.size(); ++k)
        gauss_count.push_back(ctx->h_subj_gauss_first[k + 1] - ctx->h_subj_gauss_first[k]);
    std::vector<uint8_t> frozen((size_t)M, 0);
    const bool any_frozen = ctx->any_frozen;
    if (any_frozen) CK(cudaMemcpy(frozen.data(), ctx->d_frozen.p, (size_t)M, cudaMemcpyDeviceToHost));
    DBuf<float> I;
    DBuf<uint8_t> mask;
    if (had_obs) {
        CK(I.ensure((size_t)ctx->P));
        CK(mask.ensure((size_t)ctx->P));
        CK(cudaMemcpy(I.p, ctx->d_I.p, sizeof(float) * ctx->P, cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(mask.p, ctx->d_mask.p, (size_t)ctx->P, cudaMemcpyDeviceToDevice));
    }
    gsvr_status s = gsvr_set_stacks(ctx, (int32_t)desc.size(), desc.data());
    if (!s && had_obs) s = gsvr_set_observations(ctx, I.p, mask.p, GSVR_MEM_DEVICE);
    if (!s && had_obs && ctx->have_gauss && n_subj > 1 && (int)gauss_count.size() == n_subj)
        s = gsvr_set_subjects(ctx, n_subj, stack_subject.data(), gauss_count.data());
    if (!s && any_frozen) s = gsvr_set_frozen(ctx, frozen.data());
    if (!s && ctx->have_gauss) s = ensure_item_capacity(ctx);
    if (!s) CK(cudaStreamSynchronize(ctx->stream));
    return s;
}

gsvr_status gsvr_tune_space_default(gsvr_tiling *out, int32_t cap, int32_t *n) {
    if (!n || cap < 0 || (cap > 0 && !out)) return GSVR_ERR_INVALID_ARG;
    // (tile_h, tile_w, fwd px per thread, fwd CTAs/SM, bwd CTAs/SM, queue order)
    static const int32_t space[][6] = {
        {8, 8, 0, 0, 0, 0},    {8, 8, 1, 0, 0, 0},    {12, 12, 0, 0, 0, 0},  {12, 12, 0, 0, 0, 1},
        {12, 12, 2, 0, 0, 0},  {12, 12, 0, 4, 4, 0},  {12, 12, 0, 0, -1, 0}, {12, 12, 0, -1, -1, 0},
        {16, 16, 0, 0, 0, 0},  {16, 16, 0, 0, 0, 1},  {16, 16, 2, 0, 0, 0},  {16, 16, 0, 0, -1, 0},
        {8, 16, 0, 0, 0, 0},   {16, 8, 0, 0, 0, 0},   {8, 32, 0, 0, 0, 0},   {32, 8, 0, 0, 0, 0},
        {12, 16, 0, 0, 0, 0},  {10, 10, 0, 0, 0, 0},  {10, 12, 0, 0, -1, 0}, {12, 8, 0, 0, -1, 0},
        {32, 16, 0, 0, 0, 0},  {16, 32, 0, 0, 0, 0},  {32, 32, 0, 0, 0, 0},  {16, 16, 8, 0, 0, 0}};
    const int32_t total = (int32_t)(sizeof(space) / sizeof(space[0]));
    *n = total;
    for (int32_t k = 0; k < std::min(cap, total); ++k) {
        gsvr_tiling &t = out[k];
        t.tile_h = space[k][0];
        t.tile_w = space[k][1];
        t.fwd_px_per_thread = space[k][2];
        t.fwd_blocks_per_sm = space[k][3];
        t.bwd_blocks_per_sm = space[k][4];
        t.queue_order = space[k][5];
        t.ms = 0.f;
    }
    return GSVR_OK;
}

gsvr_status gsvr_autotune(gsvr_ctx *ctx, gsvr_tiling *cand, int32_t n_cand, int64_t n_per_subject,
                          int32_t iterations, int32_t *best) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!cand || n_cand < 1 || iterations < 1 || iterations > 1000 || n_per_subject < 0)
        return fail(ctx, GSVR_ERR_INVALID_ARG, "need candidates, 1..1000 iterations, n_per_subject >= 0");
    if (!ctx->have_gauss || !ctx->have_obs) return fail(ctx, GSVR_ERR_STATE, "set stacks, observations, Gaussians first");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_autotune during graph capture");
    DeviceGuard g(ctx->device);
    const int32_t timing = ctx->cfg.timing;
    ctx->cfg.timing = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        ctx->cfg.timing = timing;
        return fail(ctx, GSVR_ERR_CUDA, "cudaEventCreate failed");
    }
    int bi = -1;
    gsvr_status hard = GSVR_OK;
    for (int32_t c = 0; c < n_cand && !hard; ++c) {
        cand[c].ms = -1.f;
        gsvr_status s = gsvr_set_tiling(ctx, &cand[c]);
        if (s == GSVR_ERR_INVALID_ARG) continue;  // not a valid launch shape: skipped
        if (s) {
            hard = s;
            break;
        }
        for (int it = 0; it <= iterations && !s; ++it) {  // iteration 0 warms up
            if (it == 1) cudaEventRecord(e0, ctx->stream);
            s = tune_iteration(ctx, n_per_subject, it);
        }
        cudaEventRecord(e1, ctx->stream);
        const gsvr_status ss = gsvr_sync_status(ctx);  // capacity / timeout flags mark the shape unusable
        if (s == GSVR_ERR_CAPACITY || ss == GSVR_ERR_CAPACITY) continue;
        if (s || ss) {
            hard = s ? s : ss;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            hard = fail(ctx, GSVR_ERR_CUDA, "event timing failed");
            break;
        }
        cand[c].ms = ms / (float)iterations;
        if (bi < 0 || cand[c].ms < cand[bi].ms) bi = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->cfg.timing = timing;
    if (hard) return hard;
    if (bi < 0) return fail(ctx, GSVR_ERR_INVALID_ARG, "no candidate launch shape ran");
    if (best) *best = bi;
    gsvr_status s = gsvr_set_tiling(ctx, &cand[bi]);
    if (s) return s;
    return GSVR_OK;
}

}  // extern "C"

// ------------------------------------------------------------- checkpoints
// File layout (host byte order, the writer's): magic "GSVRCKPT", u32 version,
// u32 section count, then sections (u32 tag, u32 0, u64 byte length, payload),
// then u64 FNV-1a hash of every byte before it.
namespace {

constexpr char kCkptMagic[8] = {'G', 'S', 'V', 'R', 'C', 'K', 'P', 'T'};
constexpr uint32_t kCkptVersion = 1;
enum : uint32_t {
    kSecConfig = 1,
    kSecGeometry = 2,
    kSecParams = 3,
    kSecStep = 4,
    kSecFrozen = 5,
    kSecObjective = 6,
    kSecSliceWeights = 7,
    kSecTopk = 8,
    kSecSubjects = 9,
    kSecDensify = 10,
    kSecCount = 10
};

uint64_t fnv1a(const unsigned char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t k = 0; k < n; ++k) {
        h ^= p[k];
        h *= 1099511628211ull;
    }
    return h;
}

struct CkptWriter {
    std::vector<unsigned char> buf;
    size_t sec_len_at = 0;
    template <class T>
    void put(const T &v) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(&v);
        buf.insert(buf.end(), b, b + sizeof(T));
    }
    void put_bytes(const void *p, size_t n) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(p);
        buf.insert(buf.end(), b, b + n);
    }
    void begin(uint32_t tag) {
        put(tag);
        put(uint32_t(0));
        sec_len_at = buf.size();
        put(uint64_t(0));
    }
    void end() {
        const uint64_t len = buf.size() - sec_len_at - sizeof(uint64_t);
        std::memcpy(&buf[sec_len_at], &len, sizeof(len));
    }
};

// One parsed checkpoint: every section's payload, validated for framing.
struct CkptFile {
    std::vector<unsigned char> data;
    const unsigned char *sec[kSecCount + 1] = {};
    uint64_t len[kSecCount + 1] = {};
};

struct CkptReader {
    const unsigned char *p;
    uint64_t n, off = 0;
    bool ok = true;
    template <class T>
    T get() {
        T v{};
        if (off + sizeof(T) > n) {
            ok = false;
            return v;
        }
        std::memcpy(&v, p + off, sizeof(T));
        off += sizeof(T);
        return v;
    }
    const unsigned char *take(uint64_t bytes) {
        if (bytes > n || off + bytes > n) {
            ok = false;
            return nullptr;
        }
        const unsigned char *q = p + off;
        off += bytes;
        return q;
    }
};

// Reads and checks the framing of a checkpoint: magic, version, hash, section
// tags (each known, at most once; config, geometry, params and step present).
std::string ckpt_read(const char *path, CkptFile &f) {
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return "cannot open checkpoint file";
    std::fseek(fp, 0, SEEK_END);
    const long sz = std::ftell(fp);
    std::fseek(fp, 0, SEEK_SET);
    if (sz < 0) {
        std::fclose(fp);
        return "cannot size checkpoint file";
    }
    f.data.resize((size_t)sz);
    const size_t got = sz > 0 ? std::fread(f.data.data(), 1, (size_t)sz, fp) : 0;
    std::fclose(fp);
    if (got != (size_t)sz) return "short read of checkpoint file";
    if (f.data.size() < 16 + sizeof(uint64_t) || std::memcmp(f.data.data(), kCkptMagic, 8) != 0)
        return "not a gsvr checkpoint (bad magic)";
    uint32_t version = 0, nsec = 0;
    std::memcpy(&version, f.data.data() + 8, 4);
    std::memcpy(&nsec, f.data.data() + 12, 4);
    if (version != kCkptVersion) return "unsupported checkpoint version " + std::to_string(version);
    const size_t body = f.data.size() - sizeof(uint64_t);
    uint64_t h = 0;
    std::memcpy(&h, f.data.data() + body, sizeof(h));
    if (h != fnv1a(f.data.data(), body)) return "checkpoint hash mismatch (truncated or corrupted file)";
    CkptReader r{f.data.data(), body, 16};
    for (uint32_t s = 0; s < nsec; ++s) {
        const uint32_t tag = r.get<uint32_t>();
        r.get<uint32_t>();
        const uint64_t len = r.get<uint64_t>();
        const unsigned char *q = r.take(len);
        if (!r.ok) return "checkpoint section runs past the end of the file";
        if (tag < 1 || tag > kSecCount || f.sec[tag]) return "unknown or repeated checkpoint section";
        f.sec[tag] = q;
        f.len[tag] = len;
    }
    if (r.off != body) return "trailing bytes after the last checkpoint section";
    for (uint32_t t : {kSecConfig, kSecGeometry, kSecParams, kSecStep})
        if (!f.sec[t]) return "checkpoint lacks a required section";
    return "";
}

struct CkptHead {
    int32_t n_stacks = 0, M = 0;
    int64_t P = 0, N = 0;
    uint64_t step = 0;
};

std::string ckpt_head(const CkptFile &f, CkptHead &h) {
    CkptReader g{f.sec[kSecGeometry], f.len[kSecGeometry]};
    h.n_stacks = g.get<int32_t>();
    h.M = g.get<int32_t>();
    h.P = g.get<int64_t>();
    if (!g.ok || h.n_stacks < 1 || h.M < 1 || h.P < 1 ||
        f.len[kSecGeometry] != 16 + (uint64_t)h.n_stacks * sizeof(gsvr_stack_desc))
        return "malformed checkpoint geometry section";
    CkptReader p{f.sec[kSecParams], f.len[kSecParams]};
    h.N = p.get<int64_t>();
    if (!p.ok || h.N < 0 || h.N > (1LL << 26) ||
        f.len[kSecParams] != 8 + 3ull * sizeof(float) * (uint64_t)(11 * h.N + 6 * (int64_t)h.M))
        return "malformed checkpoint parameter section";
    CkptReader s{f.sec[kSecStep], f.len[kSecStep]};
    h.step = s.get<uint64_t>();
    if (!s.ok || f.len[kSecStep] != 8) return "malformed checkpoint step section";
    return "";
}

}  // namespace

extern "C" {

gsvr_status gsvr_checkpoint_info(const char *path, gsvr_checkpoint_header *out, char *msg, int32_t msg_len) {
    auto say = [&](const std::string &m) {
        if (msg && msg_len > 0) {
            std::strncpy(msg, m.c_str(), (size_t)msg_len - 1);
            msg[msg_len - 1] = '\0';
        }
    };
    say("");
    if (!path || !out) {
        say("path or out is NULL");
        return GSVR_ERR_INVALID_ARG;
    }
    CkptFile f;
    std::string e = ckpt_read(path, f);
    CkptHead h;
    if (e.empty()) e = ckpt_head(f, h);
    if (!e.empty()) {
        say(e);
        return GSVR_ERR_INVALID_ARG;
    }
    out->version = (int32_t)kCkptVersion;
    out->n_stacks = h.n_stacks;
    out->n_slices = h.M;
    out->n_pixels = h.P;
    out->n_gaussians = h.N;
    out->step = (int64_t)h.step;
    return GSVR_OK;
}

gsvr_status gsvr_save(gsvr_ctx *ctx, const char *path) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!path) return fail(ctx, GSVR_ERR_INVALID_ARG, "path is NULL");
    if (!ctx->have_gauss) return fail(ctx, GSVR_ERR_STATE, "nothing to save before gsvr_set_gaussians");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_save during graph capture");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    const int M = ctx->M;
    const int64_t N = ctx->N;
    const size_t np = (size_t)(11 * N + 6 * M);
    std::vector<float> th(np), m(np), v(np);
    CK(cudaMemcpy(th.data(), ctx->d_theta.p, sizeof(float) * np, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(m.data(), ctx->d_m.p, sizeof(float) * np, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(v.data(), ctx->d_v.p, sizeof(float) * np, cudaMemcpyDeviceToHost));
    Counters cnt{};
    CK(cudaMemcpy(&cnt, ctx->d_counters.p, sizeof(Counters), cudaMemcpyDeviceToHost));
    std::vector<uint8_t> frozen((size_t)M, 0);
    if (ctx->any_frozen) CK(cudaMemcpy(frozen.data(), ctx->d_frozen.p, (size_t)M, cudaMemcpyDeviceToHost));

    CkptWriter w;
    w.put_bytes(kCkptMagic, 8);
    w.put(kCkptVersion);
    w.put(uint32_t(0));  // section count, patched below
    uint32_t nsec = 0;
    w.begin(kSecConfig);
    w.put(ctx->cfg.cutoff_rel);
    w.put(ctx->cfg.norm_mode);
    w.put(ctx->cfg.seed);
    for (int32_t x : {ctx->tile_h, ctx->tile_w, ctx->fwd_pxr_req, ctx->fwd_bps, ctx->bwd_bps, ctx->queue_order})
        w.put(x);
    w.end();
    ++nsec;
    w.begin(kSecGeometry);
    w.put((int32_t)ctx->n_stacks);
    w.put((int32_t)M);
    w.put((int64_t)ctx->P);
    w.put_bytes(ctx->h_stack_desc.data(), sizeof(gsvr_stack_desc) * ctx->h_stack_desc.size());
    w.end();
    ++nsec;
    w.begin(kSecParams);
    w.put((int64_t)N);
    w.put_bytes(th.data(), sizeof(float) * np);
    w.put_bytes(m.data(), sizeof(float) * np);
    w.put_bytes(v.data(), sizeof(float) * np);
    w.end();
    ++nsec;
    w.begin(kSecStep);
    w.put((uint64_t)cnt.step);
    w.end();
    ++nsec;
    w.begin(kSecFrozen);
    w.put_bytes(frozen.data(), frozen.size());
    w.end();
    ++nsec;
    w.begin(kSecObjective);
    w.put((int32_t)ctx->loss_kind);
    w.put(ctx->lambda_reg);
    w.put(ctx->s_target);
    w.end();
    ++nsec;
    w.begin(kSecSliceWeights);
    w.put((int32_t)(ctx->slw_on ? 1 : 0));
    w.put(ctx->lr_slw_sig);
    w.put(ctx->lr_slw_omg);
    if (ctx->slw_on) {
        std::vector<float> sp(2 * (size_t)M);
        for (DBuf<float> *b : {&ctx->d_slw, &ctx->d_slw_m, &ctx->d_slw_v}) {
            CK(cudaMemcpy(sp.data(), b->p, sizeof(float) * sp.size(), cudaMemcpyDeviceToHost));
            w.put_bytes(sp.data(), sizeof(float) * sp.size());
        }
    }
    w.end();
    ++nsec;
    w.begin(kSecTopk);
    w.put((int32_t)ctx->topk_K);
    w.put((int32_t)ctx->topk_refresh);
    w.put(ctx->topk_delta);
    w.put(ctx->topk_per_cell);
    w.end();
    ++nsec;
    w.begin(kSecSubjects);
    w.put((int32_t)ctx->n_subj);
    if (ctx->n_subj > 1) {
        w.put_bytes(ctx->h_stack_subject.data(), sizeof(int) * (size_t)ctx->n_stacks);
        w.put_bytes(ctx->h_subj_gauss_first.data(), sizeof(int64_t) * ((size_t)ctx->n_subj + 1));
    }
    w.put((int32_t)ctx->h_subj_active.size());
    w.put_bytes(ctx->h_subj_active.data(), ctx->h_subj_active.size());
    w.end();
    ++nsec;
    w.begin(kSecDensify);
    const int64_t dn = (ctx->dens_n == N && ctx->d_dens_acc.p && ctx->d_dens_cnt.p) ? N : -1;
    w.put(dn);
    if (dn >= 0) {
        std::vector<float4> acc((size_t)std::max<int64_t>(N, 1));
        int c = 0;
        CK(cudaMemcpy(acc.data(), ctx->d_dens_acc.p, sizeof(float4) * acc.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&c, ctx->d_dens_cnt.p, sizeof(int), cudaMemcpyDeviceToHost));
        w.put_bytes(acc.data(), sizeof(float4) * (size_t)N);
        w.put((int32_t)c);
    }
    w.end();
    ++nsec;
    std::memcpy(&w.buf[12], &nsec, sizeof(nsec));
    const uint64_t h = fnv1a(w.buf.data(), w.buf.size());
    w.put(h);

    // written to a temporary name, then renamed over `path`
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) return fail(ctx, GSVR_ERR_INVALID_ARG, "cannot open checkpoint file for writing");
    const size_t put = std::fwrite(w.buf.data(), 1, w.buf.size(), fp);
    const int cl = std::fclose(fp);
    if (put != w.buf.size() || cl != 0 || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(ctx, GSVR_ERR_INVALID_ARG, "writing the checkpoint file failed");
    }
    return GSVR_OK;
}

gsvr_status gsvr_load(gsvr_ctx *ctx, const char *path) {
    if (check_ctx(ctx)) return GSVR_ERR_INVALID_ARG;
    if (!path) return fail(ctx, GSVR_ERR_INVALID_ARG, "path is NULL");
    if (!ctx->have_stacks || !ctx->have_obs)
        return fail(ctx, GSVR_ERR_STATE, "gsvr_set_stacks and gsvr_set_observations before gsvr_load");
    if (ctx->capturing) return fail(ctx, GSVR_ERR_STATE, "gsvr_load during graph capture");
    CkptFile f;
    std::string e = ckpt_read(path, f);
    CkptHead hd;
    if (e.empty()) e = ckpt_head(f, hd);
    if (!e.empty()) return fail(ctx, GSVR_ERR_INVALID_ARG, e);
    // the context must hold the same acquisition (stacks compared byte for byte)
    if (hd.n_stacks != ctx->n_stacks || hd.M != ctx->M || hd.P != ctx->P ||
        std::memcmp(f.sec[kSecGeometry] + 16, ctx->h_stack_desc.data(),
                    sizeof(gsvr_stack_desc) * (size_t)ctx->n_stacks) != 0)
        return fail(ctx, GSVR_ERR_STATE, "checkpoint stacks differ from the context's");
    const int M = ctx->M;
    const int64_t N = hd.N;
    const size_t np = (size_t)(11 * N + 6 * M);
    // parse every optional section before changing anything
    CkptReader rc{f.sec[kSecConfig], f.len[kSecConfig]};
    const float cutoff = rc.get<float>();
    const int32_t norm_mode = rc.get<int32_t>();
    const uint64_t seed = rc.get<uint64_t>();
    gsvr_tiling tl{};
    tl.tile_h = rc.get<int32_t>();
    tl.tile_w = rc.get<int32_t>();
    tl.fwd_px_per_thread = rc.get<int32_t>();
    tl.fwd_blocks_per_sm = rc.get<int32_t>();
    tl.bwd_blocks_per_sm = rc.get<int32_t>();
    tl.queue_order = rc.get<int32_t>();
    if (!rc.ok || rc.off != rc.n || !(cutoff > 0.f && cutoff < 1.f) ||
        (norm_mode != GSVR_NORM_EXACT && norm_mode != GSVR_NORM_LITERAL))
        return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed checkpoint config section");
    if (gsvr_status s = check_tiling(ctx, tl)) return s;
    // the payload is copied out: sections follow one another at any byte offset
    std::vector<float> th(3 * np);
    std::memcpy(th.data(), f.sec[kSecParams] + 8, sizeof(float) * th.size());
    std::vector<uint8_t> frozen((size_t)M, 0);
    if (f.sec[kSecFrozen]) {
        if (f.len[kSecFrozen] != (uint64_t)M) return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed frozen section");
        std::memcpy(frozen.data(), f.sec[kSecFrozen], (size_t)M);
    }
    int32_t loss_kind = 0;
    float lambda_reg = 0.f, s_target = 1.6f;
    if (f.sec[kSecObjective]) {
        CkptReader r{f.sec[kSecObjective], f.len[kSecObjective]};
        loss_kind = r.get<int32_t>();
        lambda_reg = r.get<float>();
        s_target = r.get<float>();
        if (!r.ok || r.off != r.n) return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed objective section");
    }
    int32_t slw_on = 0;
    float lr_sig = 1e-3f, lr_omg = 1e-2f;
    std::vector<float> slw;
    if (f.sec[kSecSliceWeights]) {
        CkptReader r{f.sec[kSecSliceWeights], f.len[kSecSliceWeights]};
        slw_on = r.get<int32_t>();
        lr_sig = r.get<float>();
        lr_omg = r.get<float>();
        if (slw_on) {
            const unsigned char *q = r.take(3ull * 2 * sizeof(float) * (uint64_t)M);
            if (q) {
                slw.resize(6 * (size_t)M);
                std::memcpy(slw.data(), q, sizeof(float) * slw.size());
            }
        }
        if (!r.ok || r.off != r.n) return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed slice-weight section");
    }
    int32_t topk_K = 0, topk_refresh = 1;
    float topk_delta = 1e-8f, topk_per_cell = 16.f;
    if (f.sec[kSecTopk]) {
        CkptReader r{f.sec[kSecTopk], f.len[kSecTopk]};
        topk_K = r.get<int32_t>();
        topk_refresh = r.get<int32_t>();
        topk_delta = r.get<float>();
        topk_per_cell = r.get<float>();
        if (!r.ok || r.off != r.n || !(topk_per_cell > 0.f))
            return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed top-K section");
    }
    int32_t n_subj = 1, n_active = 0;
    std::vector<int32_t> stack_subject;
    std::vector<int64_t> gauss_count;
    std::vector<uint8_t> active;
    if (f.sec[kSecSubjects]) {
        CkptReader r{f.sec[kSecSubjects], f.len[kSecSubjects]};
        n_subj = r.get<int32_t>();
        if (n_subj > 1 && n_subj <= 65536) {
            stack_subject.resize((size_t)ctx->n_stacks);
            std::vector<int64_t> gf((size_t)n_subj + 1);
            const unsigned char *a = r.take(sizeof(int32_t) * stack_subject.size());
            const unsigned char *b = r.take(sizeof(int64_t) * gf.size());
            if (a && b) {
                std::memcpy(stack_subject.data(), a, sizeof(int32_t) * stack_subject.size());
                std::memcpy(gf.data(), b, sizeof(int64_t) * gf.size());
                for (int k = 0; k < n_subj; ++k) gauss_count.push_back(gf[(size_t)k + 1] - gf[(size_t)k]);
            }
        }
        n_active = r.get<int32_t>();
        if (n_active > 0 && n_active == n_subj) {
            const unsigned char *a = r.take((uint64_t)n_active);
            if (a) active.assign(a, a + n_active);
        } else if (n_active != 0) {
            r.ok = false;
        }
        if (!r.ok || r.off != r.n || n_subj < 1 || n_subj > 65536)
            return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed subject section");
    }
    int64_t dens_n = -1;
    std::vector<float4> dens_acc;
    int32_t dens_cnt = 0;
    if (f.sec[kSecDensify]) {
        CkptReader r{f.sec[kSecDensify], f.len[kSecDensify]};
        dens_n = r.get<int64_t>();
        if (dens_n >= 0) {
            if (dens_n != N) r.ok = false;
            else if (const unsigned char *q = r.take(sizeof(float4) * (uint64_t)N)) {
                dens_acc.resize((size_t)std::max<int64_t>(N, 1));
                std::memcpy(dens_acc.data(), q, sizeof(float4) * (size_t)N);
            }
            dens_cnt = r.get<int32_t>();
        }
        if (!r.ok || r.off != r.n) return fail(ctx, GSVR_ERR_INVALID_ARG, "malformed densification section");
    }

    // apply: configuration and launch shape, parameters, then the optimiser state
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    drop_graph(ctx);
    ctx->cfg.cutoff_rel = cutoff;
    ctx->cfg.norm_mode = norm_mode;
    ctx->cfg.seed = seed;
    ctx->rc2 = (float)(2.0 * std::log(1.0 / (double)cutoff));
    if (gsvr_status s = gsvr_set_tiling(ctx, &tl)) return s;
    if (gsvr_status s = gsvr_set_gaussians(ctx, N, th.data(), GSVR_MEM_HOST)) return s;
    if (n_subj > 1) {
        if (gsvr_status s = gsvr_set_subjects(ctx, n_subj, stack_subject.data(), gauss_count.data())) return s;
    } else if (ctx->n_subj != 1) {
        if (gsvr_status s = gsvr_set_subjects(ctx, 1, nullptr, nullptr)) return s;
    }
    if (!active.empty())
        if (gsvr_status s = gsvr_set_subject_active(ctx, active.data())) return s;
    if (gsvr_status s = gsvr_set_frozen(ctx, frozen.data())) return s;
    if (gsvr_status s = gsvr_set_objective(ctx, loss_kind, lambda_reg, s_target)) return s;
    if (gsvr_status s = gsvr_set_slice_weights(ctx, slw_on, lr_sig, lr_omg)) return s;
    ctx->topk_per_cell = topk_per_cell;
    if (gsvr_status s = gsvr_set_topk(ctx, topk_K, topk_delta, topk_refresh)) return s;
    // parameters, Adam moments and step counter exactly as saved
    CK(cudaMemcpy(ctx->d_theta.p, th.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_m.p, th.data() + np, sizeof(float) * np, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_v.p, th.data() + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice));
    if (!slw.empty()) {
        const size_t n2 = 2 * (size_t)M;
        CK(cudaMemcpy(ctx->d_slw.p, slw.data(), sizeof(float) * n2, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_slw_m.p, slw.data() + n2, sizeof(float) * n2, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_slw_v.p, slw.data() + 2 * n2, sizeof(float) * n2, cudaMemcpyHostToDevice));
    }
    if (!dens_acc.empty()) {
        if (gsvr_status s = dens_ensure(ctx)) return s;
        CK(cudaMemcpy(ctx->d_dens_acc.p, dens_acc.data(), sizeof(float4) * (size_t)N, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_dens_cnt.p, &dens_cnt, sizeof(int), cudaMemcpyHostToDevice));
    }
    if (gsvr_status s = gsvr_set_step(ctx, (int64_t)hd.step)) return s;
    ctx->fwd_valid = false;
    return GSVR_OK;
}

}  // extern "C"
