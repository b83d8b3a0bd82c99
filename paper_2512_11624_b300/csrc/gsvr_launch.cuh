// gsvr_launch.cuh -- argument blocks and host launchers of the libgsvr kernels.
#pragma once
#include "gsvr_internal.cuh"

namespace gsvr {

struct BinArgs {
    const float *theta;        // 11N + 6M
    const float4 *gpre;        // 2 per Gaussian: (Sxx, Syy, Szz, Sxy), (Sxz, Syz, sum ls, c)
    const SliceDev *slices;
    int N, M;
    float rc2;                 // squared Mahalanobis cut: 2 ln(1 / cutoff_rel)
    int norm_mode;
    int tile_w, tile_h;
    float qcut;                // log2(cutoff_rel): per-pair exponent cut (log2 units)
    const int *tile_px_start, *tile_px_end;
    int *rec_cnt;              // candidates per Gaussian (count pass)
    const int *rec_off;        // first candidate of each Gaussian, N + 1
    const int *n_rec;          // device count of candidates (= records)
    int2 *cand;                // (Gaussian, slice) per candidate; slice -1 = padding
    unsigned *cand_mask;       // slab-test bits of the count pass, word w of Gaussian j at [w * N + j]
                               // (ceil(M / 32) words; null or a multi-subject batch: the emit pass tests again)
    const int *gauss_subject;  // subject of each Gaussian (null: one subject)
    const int *subj_slice_first;  // first slice of each subject (n_subj + 1)
    const uint8_t *subj_active;   // per subject, 0 = retired: its Gaussians meet no slice (null: all active)
    Rec *rec;                  // one record per candidate
    int2 *rec_tiles;           // packed tile bounding box per record
    int *rec_nkeys;            // keys per record
    unsigned *rec_mask;        // live tiles of the box, row-major bits (0 when the box exceeds 32 tiles)
    int cap_rec;
    unsigned *status;
};

struct KeyArgs {
    const Rec *rec;
    const int2 *cand;          // (Gaussian, slice) per record
    const int2 *rec_tiles;
    const int *rec_nkeys;      // keys per record (from the record pass)
    const unsigned *rec_mask;  // live-tile bits of the record pass (0: test again)
    const int *key_off;        // n_rec + 1
    const SliceDev *slices;
    const int *tile_px_start, *tile_px_end;
    const int *n_rec;          // device count
    int cap_rec, cap_keys;
    int tile_w, tile_h, n_tiles;
    float qcut;
    uint32_t *keys;
    int *key_rec;
    float4 *mom;               // backward moments: zeroed here for padding (sentinel) keys
    unsigned *status;
};

struct EvalArgs {
    const int2 *tref;          // per sorted key: (record, emit index); capacity + 2 entries
    const Rec *rec;            // records, Gaussian-major
    const int *tile_rec_start, *tile_rec_end;
    const int *tile_px_start, *tile_px_end;
    const int *tile_slice;
    const SliceDev *slices;
    const int *sampled;        // global pixel index, tile order
    const int *n_sampled;
    const float *I_obs;        // per global pixel
    float *pred, *rbar;        // per global pixel
    int *tpos_s;               // tile-local (row << 8 | col) per sample position (null: not written)
    short2 *row_rng;           // per tile row: sampled columns (lo, hi; lo > hi: none), from k_fwd_reduce (null: not written)
    float *rbar_tile;          // dense r_bar per tile pixel (0 off the sample), built before the backward
    const int *pix_tile;       // tile of each global pixel
    double *tile_loss;         // per tile
    float4 *mom;               // 2 per key (backward)
    Counters *counters;
    unsigned long long *pairs_total;  // running sum of visited pairs (timing)
    unsigned long long *bwd_pairs_total;  // running sum of pairs the backward evaluated (null: not counted)
    unsigned long long *useful;       // count mode: pairs inside the cut
    float qcut;                       // count mode: log2(cutoff_rel)
    const int *item_tile;             // tile of each work item
    const int *item_first;            // first item of each tile (n_tiles + 1)
    const int *n_items;               // device count
    float *part;                      // per-item partial pixel sums (cap_items x tile_px)
    int cap_items;
    const int *subj_cnt;              // sampled pixels per subject (null: *n_sampled)
    const uint32_t *item_order;       // work-queue order of the items (null: item index order)
    int fwd_pxr;                      // forward pixels per thread, 1, 2, 4, 8 or 16 (0: by tile width)
    int fwd_bps, bwd_bps;             // persistent CTAs per SM (0: as many as fit)
    int tile_px;                      // tile_w * tile_h
    int l1;                           // data term: 0 MSE, 1 L1 (the paper's)
    const float *slw;                 // per-slice log sigma_i (M) then log omega_i (M), or null
    double *slw_gacc;                 // their gradients (2 M)
    double *slw_tile;                 // per tile: the tile's terms of the two (2 per tile, plain forward)
    int M;
    int tile_w, tile_h;
    int n_tiles;
    unsigned *status;
    int64_t n_weight;                 // > 0: pixel weight 1 / n_weight (gsvr_set_sample_total), else 1 / sample size
    // test hook (gsvr_test_wait_timeout): > 0 makes every block's first record
    // wait of the forward wait, bounded by this many ns, on a barrier nothing completes
    int64_t wait_test_ns;
};

struct GradArgs {
    const float *theta;
    const float4 *gpre;
    const SliceDev *slices;
    const Rec *rec;            // j-major records, slot b.w = slice index
    const int *rec_off;        // N + 1
    const int2 *cand;          // (Gaussian, slice) per record
    const int *key_off;        // n_rec + 1
    const float4 *mom;         // 2 per key in emit order
    const uint32_t *keys;      // tile id per key in emit order (n_tiles = sentinel)
    int n_tiles;
    int N, M;
    float rc2;
    int norm_mode;
    float *grad;               // 11N + 6M
    double *pose_acc;          // M x 12: dL/dR_i (9), dL/dt_i (3)
    const int *gauss_subject;  // subject of each Gaussian (null: one subject)
    const int *subj_slice_first;
    int smem_slices;           // slice window that fits the shared accumulators (0: none)
    int smem_geo;              // the window's slice geometry is staged in shared memory too (set by the launcher)
    // host copies of the subject tables (n_subj + 1 entries each), used by the
    // launcher to size the shared window
    const int64_t *h_gauss_first;
    const int *h_slice_first;
    int n_subj;
    int cap_rec, cap_keys;     // reads stay inside the buffers even after an overflow
};

void launch_gauss_prep(const float *theta, int N, float4 *gpre, unsigned *status, cudaStream_t st);
void launch_pose_prep(const float *pose, const SliceStatic *ss, SliceDev *sd, int M, unsigned *status,
                      cudaStream_t st);
void launch_cand_count(const BinArgs &a, cudaStream_t st);
void launch_cand_emit(const BinArgs &a, cudaStream_t st);
void launch_records(const BinArgs &a, int n_cand_max, cudaStream_t st);
void launch_key_emit(const KeyArgs &a, int n_rec_max, cudaStream_t st);
void launch_tile_rec_ranges(const uint32_t *keys, const int *n_keys, int cap_keys, int n_tiles, int *start, int *end,
                            cudaStream_t st);
// phase 0: items per tile into cnt; phase 1: item -> tile from the scanned offsets `first`
void launch_items(const int *tps, const int *tpe, const int *trs, const int *tre, int n_tiles, int *cnt,
                  const int *first, int *item_tile, int cap_items, int phase, cudaStream_t st,
                  unsigned long long *pairs = nullptr, unsigned long long *pairs_total = nullptr);
void launch_forward(const EvalArgs &a, cudaStream_t st);
void launch_count_pairs(const EvalArgs &a, cudaStream_t st);
long long launch_count();  // kernels launched by this library so far
void note_launches(int n); // count kernels launched from other translation units
// Dense r_bar tiles (from the per-pixel r_bar of the cap_px sample slots), then the tile adjoint.
void launch_backward(const EvalArgs &a, int cap_px, cudaStream_t st);
// Per-subject losses (subject k owns tiles [tile_first[k], tile_first[k+1]), summed in
// tile order) and their total; tile_first null = one subject.
void launch_loss_reduce(const double *tile_loss, int n_tiles, const int *tile_first, int n_subj, double *subj_loss,
                        double *loss, unsigned *status, cudaStream_t st);
// Sampled pixels per subject: cnt[k] = sum of the subject's tile pixel counts.
void launch_subject_counts(const int *tps, const int *tpe, const int *tile_first, int n_subj, int *cnt,
                           cudaStream_t st);
// Occupancy of the evaluation kernels (blocks per SM) for the persistent grids.
int eval_blocks_per_sm(int tile_w, int tile_h, bool backward, int fwd_pxr_req);
int fwd_pxr(int tile_w, int req);
int fwd_threads(int tile_w, int tile_h, int pxr);
bool fwd_shape_fits(int tile_w, int tile_h, int pxr);  // the groups' per-pixel sums fit the forward's shared buffer
// Work-queue order: items sorted by descending record count (stable).
void launch_item_order(const int *item_tile, const int *item_first, const int *trs, const int *tre,
                       const int *n_items, int cap_items, uint32_t *key, uint32_t *key_sorted, uint32_t *order,
                       const SortScratch &ss, cudaStream_t st);
void launch_gauss_grad(const GradArgs &a, cudaStream_t st);
void launch_pose_grad(const double *pose_acc, const SliceStatic *ss, const float *pose, float *grad_pose, int M,
                      cudaStream_t st);
// Adam with StepLR (lr x gamma^((t-1) / step_every), step_every 0 = constant); the
// 1-based step t comes from `t_host` or, when d_step is non-null, from *d_step + 1.
void launch_adam(float *theta, const float *grad, float *m, float *v, int N, int M, const float lr[6], float b1,
                 float b2, float eps, int step_every, float gamma, long long t_host, const unsigned long long *d_step,
                 float *d_scal, const uint8_t *frozen, cudaStream_t st);
void launch_advance_step(unsigned long long *d_step, cudaStream_t st);
// Adam on the per-slice terms (2 M: log sigma_i with lr_sig, log omega_i with
// lr_omg), same schedule and step as launch_adam (call it after launch_adam,
// whose device scalars it reads when d_step is given); frozen slices keep
// their sigma (the intensity gauge), not their omega.
void launch_adam_slw(float *p, const float *g, float *m, float *v, int M, float lr_sig, float lr_omg, float b1,
                     float b2, float eps, int step_every, float gamma, long long t_host, const unsigned long long *d_step,
                     const float *d_scal, const uint8_t *frozen, cudaStream_t st);
// ---- content-adaptive initialisation of the means (Sec. 2.5)
// W[p] = floor(1024 ((1 - lam) |grad I_p| + lam)) over masked pixels (0
// elsewhere), the gradient in float32 with every operation rounded alone;
// C = inclusive prefix sum of W (int64, `scratch` >= cdiv(P, 4096) + 1 entries).
void launch_init_weights(const float *I, const uint8_t *mask, const SliceDev *slices, int M, int64_t P, float lam,
                         int64_t *W, int64_t *C, int64_t *scratch, cudaStream_t st);
// Draw k: pixel = first p with C[p] > floor(splitmix64(seed, k) T / 2^64), T =
// C[P-1]; mean = that pixel's world position jittered by uniforms from
// splitmix64(seed, 2^40 + 3 k + a) within its voxel (dx, dy, thickness).
void launch_init_draw(const int64_t *C, int64_t P, uint64_t seed, int64_t n, const SliceDev *slices, int M,
                      const float *thickness, float *mu, int *pix, cudaStream_t st);
// float copy of the forward's float64 per-slice gradient sums
void launch_slw_grad(const double *gacc, int n, float *grad, cudaStream_t st);
// gacc[i], gacc[M + i] = slice i's per-tile terms (slw_tile) summed in tile order
void launch_slw_slices(const double *slw_tile, const SliceDev *slices, int M, double *gacc, cudaStream_t st);

// Sampler: for subject k, out_first[k+1] - out_first[k] of its mask_count[k]
// masked pixels (tile-order positions mask_tpos[mask_first[k] + x]); the round
// keys come from SplitMix64(seed + k * golden gamma, 4 step + r), the step from
// `step` or, when d_step is non-null, from *d_step.
void launch_sample_flags(int n_subj, const int *mask_first, const int *out_first, int n_out, uint64_t seed,
                         uint64_t step, const unsigned long long *d_step, const int *mask_tpos, int *flags,
                         cudaStream_t st);
void launch_flags_from_list(const int *idx, int n, int n_pix, const uint8_t *mask, const int *pix_tpos,
                            int *flags, unsigned *status, cudaStream_t st);
void launch_flags_from_list_rank(const int *idx, int n, int n_pix, const int *pix_mrank, int *flags,
                                 unsigned *status, cudaStream_t st);
void launch_compact(const int *flags, const int *pos, const int *tile_sorted_pix, int n_pix, int *sampled,
                    cudaStream_t st);
void launch_tile_px_ranges(const int *sampled, const int *n_sampled, int cap, const int *pix_tile, int *start,
                           int *end, cudaStream_t st);
void launch_set_count(int *dst, int v, cudaStream_t st);

// ---- normalised top-K forward (Eq. 2 with Sigma_obs, Eq. 5 ratio; Sec. 2.5 Top-K)
// Uniform grid over the Gaussian means: cell size from the means' bounding box
// so that a cell holds about `per_cell` means, at most `max_cells` cells.
struct TopkGrid {
    float org[3];
    float h, inv_h;
    int n[3];
    int n_cells;
    int box[6];  // order-preserving integer images of the means' min (xyz) and max (xyz)
};
constexpr int kTopkMaxK = 128;
constexpr int kTopkThreads = 128;
constexpr int kTopkMaxCells = 1 << 16;
struct TopkArgs {
    const float *theta;      // 11 N + 6 M (means and amplitudes read here)
    const float4 *gpre;      // Sigma_j and c per Gaussian (k_gauss_prep)
    const SliceDev *slices;
    int N, M;
    const int *sampled;      // sampled global pixels
    const int *n_sampled;
    const float *I_obs;
    float *pred, *rbar;
    float2 *pstat;           // per sample: (I_hat, sum E + delta)
    int *nbr;                // per sample: K Gaussian indices
    int *ncnt;               // per sample: neighbours found (< K only when N < K)
    double *loss_part;       // per forward block
    const TopkGrid *grid;
    const int *cell_start, *cell_end;
    const uint32_t *gidx;    // Gaussian indices in cell order
    const float4 *gm;        // (mu, Gaussian index) in cell order, as of the last grid build
    float *gacc;             // 10 x N: d mu (3), d Sigma (xx yy zz xy xz yz), d c
    double *pose_acc;        // M x 12
    int K;
    float delta;
    int cap_px;
    int l1;                  // data term: 0 MSE, 1 L1
    const float *slw;        // per-slice log sigma_i, log omega_i (2 M) or null
    double *slw_gacc;        // their gradients (2 M)
    int64_t n_weight;        // > 0: pixel weight 1 / n_weight, else 1 / sample size
    unsigned *status;
};
// Grid build: bounding box, cell size, cell keys; the caller sorts the keys
// (stable radix, Gaussian index as value) and calls launch_topk_cell_ranges.
void launch_topk_grid(const float *theta, int N, float per_cell, TopkGrid *g, uint32_t *keys, cudaStream_t st);
void launch_topk_cell_ranges(const uint32_t *keys_sorted, int N, int *cell_start, int *cell_end, cudaStream_t st);
// gm[k] = (mu of Gaussian gidx[k], gidx[k] as float bits): the search reads one 16-byte record per candidate
void launch_topk_gather_means(const float *theta, const uint32_t *gidx, int N, float4 *gm, cudaStream_t st);
// Forward: K nearest by a shell search of the grid, the ratio per sampled
// pixel, residuals and per-block loss partials; then the loss total.
void launch_topk_forward(const TopkArgs &a, int cap_px, double *loss, cudaStream_t st);
// Backward: per (pixel, neighbour) gradients summed per block in shared memory
// (Gaussians by hashing, slices by a small table), then added to gacc and
// pose_acc; the Gaussian epilogue maps gacc to the parameter gradient.
void launch_topk_backward(const TopkArgs &a, int cap_px, cudaStream_t st);
void launch_topk_epilogue(const float *theta, const float *gacc, int N, float *grad, cudaStream_t st);

// Scale regulariser of the paper's loss (Sec. 2.5): lambda sum_j sum_k
// (exp(ls_jk) - s_target)^2 added to *loss (one block, fixed order), and its
// gradient 2 lambda (s - s_target) s added to the log-scale gradients.
void launch_scale_reg_loss(const float *theta, int N, float lambda, float s_target, double *loss, cudaStream_t st);
void launch_scale_reg_grad(const float *theta, int N, float lambda, float s_target, float *grad, cudaStream_t st);

// densification (split / clone / prune)
enum : int { kDensPrune = 0, kDensKeep = 1, kDensSplit = 2, kDensClone = 3 };
struct DensParams {
    float split_factor;      // phi
    float log_split_factor;  // ln phi
    float split_offset;      // sqrt(1 - 1 / phi^2)
    float clone_offset;      // kappa
    int mass_preserving;
};
void launch_dens_accum(const float *grad, int N, float4 *acc, int *cnt, cudaStream_t st);
void launch_dens_decide(const float *theta, int N, const float4 *acc, const int *cnt, float tau_g, float tau_ls,
                        float eps_c, uint8_t *kind, int *nout, int *counts, cudaStream_t st);
void launch_dens_emit(const float *theta, const float *m, const float *v, int N, const float4 *acc,
                      const uint8_t *kind, const int *off, int N2, const DensParams &p, float *theta2, float *m2,
                      float *v2, cudaStream_t st);

}  // namespace gsvr
