// Internal declarations of the CUDA rasterizer: the per-Gaussian record, the
// workspace layout and the launch helpers of each translation unit.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kTile = GS_TILE;
constexpr int kTilePix = kTile * kTile;        // 256 pixels, one thread each
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                  // items per thread per round-trip
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxSortBlocks = 1024;           // histogram rows reserved in the workspace
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 0x1.010102p-8f;    // 1/255 rounded to float
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;              // EWA low-pass filter added to the 2D covariance (px^2)
constexpr float kFrustumClamp = 1.3f;          // x/z and y/z clamped to this multiple of the half field of view
constexpr float kRadiusSigmas = 3.0f;          // splat radius in standard deviations of the larger eigenvalue
constexpr float kEigenFloor = 0.1f;            // floor of (mid^2 - det) under the eigenvalue square root
constexpr uint32_t kSeg = 256;                 // list positions per backward segment (checkpoint stride)
constexpr int kCbMaxDim = 48;                  // SH codebook: coordinates per row, 3(K-1) <= 45 padded
constexpr int kBinMaxDim = 256;                // tile rows and columns the binning handles (4096 px)
constexpr int kBinBlocks = 256;                // CTAs (of 8 chunk warps) of the row pass of the binning
constexpr int kBinChunks = kBinBlocks * 8;     // chunks of the depth order in the row pass
constexpr int kBinChunksPerThread = kBinChunks / 1024;

// Per-Gaussian record written by the preprocess and gathered by the compositor.
// a = (u, v, A2, beta), b = (G2, opacity, r, g), c = (b, depth, rect01, rect23)
// where the splat exponent in base 2 is A2 (dx + beta dy)^2 + G2 dy^2,
// rect01 = x0 | y0 << 16 and rect23 = x1 | y1 << 16 (half-open tile rectangle).
struct __align__(16) Rec {
    float4 a;
    float4 b;
    float4 c;
};

// Device control block at offset 0 of the workspace.  The first member is
// the public gs_status; the rest are counts the kernels hand to each other.
struct Ctl {
    gs_status st;          // 32 bytes
    uint32_t n_vis;        // visible Gaussians (counted by the depth-sort histograms)
    uint32_t dbg_site;     // GS_DEBUG builds: number of the first failed bounds check (0: none)
    uint32_t depth_mm[2];  // ~min and max of the visible depth keys (digits the sort can skip)
    uint32_t fwd_queue;    // next work item of the persistent forward compositor
    uint32_t bwd_queue;    // next work item of the persistent backward compositor
    uint32_t n_items;      // backward work items (tile, 8x8 block, segment)
    uint32_t n_pieces;     // row-list pieces of the binning
    uint32_t sort_ticket[4];   // next tile of each digit kernel of the depth sort (after the first)
    uint32_t bin_scan_done;    // CTAs of the binning's per-row scan that have finished (the last one finishes)
    uint32_t pad[11];
};
static_assert(sizeof(Ctl) == 128, "Ctl layout");

// Bounds checks of GS_DEBUG builds.  GS_CHECK(ok, ctl, site) is `ok` in a
// debug build, where a false `ok` also sets GS_ERR_BOUNDS in the status word
// (unless an error is already there) and the site number of the first failed
// check; callers skip the access when it is false.  In release builds it is
// the constant true and the check compiles away.  Site numbers:
enum DebugSite : uint32_t {
    kSiteRect = 1,          // preprocess: tile rectangle inside the tile grid
    kSiteSortScatter = 2,   // depth sort: scatter position below the item count
    kSiteRowList = 3,       // binning: row-list position below the pair capacity
    kSitePairList = 4,      // binning: pair-list position below the pair capacity
    kSiteRange = 5,         // binning: tile range inside the pair count
    kSiteFwdId = 6,         // forward compositor: Gaussian id from the list below n
    kSiteCkpt = 7,          // forward compositor: checkpoint segment inside the checkpoint area
    kSiteBwdId = 8,         // backward compositor: Gaussian id from the list below n
};
#ifdef GS_DEBUG
__device__ __forceinline__ bool gs_check(bool ok, const Ctl *ctl, uint32_t site) {
    if (!ok) {
        Ctl *c = const_cast<Ctl *>(ctl);
        atomicCAS(reinterpret_cast<int *>(&c->st.error), GS_OK, GS_ERR_BOUNDS);
        atomicCAS(&c->dbg_site, 0u, site);
    }
    return ok;
}
#define GS_CHECK(ok, ctl, site) ::gs::gs_check((ok), (ctl), (site))
#else
#define GS_CHECK(ok, ctl, site) true
#endif

// Workspace carve-up.  Every region starts on a 256-byte boundary.
struct Layout {
    int64_t n = 0, dup_cap = 0;
    int W = 0, H = 0, Tx = 0, Ty = 0, Tn = 0;
    uint32_t bin_piece = 0;
    size_t ctl = 0, rec = 0, tiles = 0, depth = 0, sort_k[2] = {0, 0}, sort_v[2] = {0, 0}, order = 0, vis_index = 0,
           sort_hist = 0, sort_grp = 0, sort_cnt = 0, sort_status = 0, bin_m = 0,
           bin_rows = 0, bin_p = 0, rowlist = 0, list = 0, ranges = 0, t_final = 0, n_contrib = 0,
           partials = 0, rec_grad = 0, tile_order = 0, qdone = 0, seg_base = 0, qwork = 0,
           ckpt = 0, items = 0, total = 0;
};

// Returns false when sizes overflow.
bool make_layout(int64_t n, int W, int H, int64_t dup_cap, Layout *L);
// Largest duplicate capacity that fits in ws_bytes (0 if even the fixed part does not fit).
int64_t capacity_for(int64_t n, int W, int H, size_t ws_bytes);

template <typename T>
inline T *at(void *base, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(base) + off); }

// Halves per row of an SH codebook table: 3(K-1) rounded up to 8 (16-byte rows).
__host__ __device__ constexpr int cb_row_halves(int K) { return (3 * (K - 1) + 7) / 8 * 8; }

struct SceneView {
    const uint16_t *sh_index;   // codebook storage: index per Gaussian
    const void *sh_table;       // codebook storage: FP16 rows of cb_row_halves(K)
    int sh_table_rows;
    const float *means;
    const void *log_scales;
    const void *quats;
    const float *opacity_logit;
    const void *sh;
    const uint8_t *layer;
    int n;
    int sh_degree;
    int dtype_sh;
    int dtype_sr;
};

struct CamView {
    float R[9];
    float t[3];
    float fx, fy, cx, cy, znear;
    int W, H, Tx, Ty;
};

struct Planes {
    float4 p[GS_MAX_PLANES];
    uint32_t bits[GS_MAX_PLANES];
    int n;
};

// ---- launches (each returns cudaGetLastError() of its launches) ----
cudaError_t launch_preprocess(const SceneView &s, const CamView &c, uint32_t layer_mask, const Planes &pl,
                              Rec *rec, uint32_t *tiles, uint32_t *depth_key, const Ctl *ctl, cudaStream_t st);
// Also adds the per-Gaussian blend-weight sums (record-gradient slot 9) to
// contrib_sum when it is not null.
// vis_index: the visible list of the last render (index order, ctl->n_vis
// entries; a two-eye list may also hold Gaussians this view does not see).
cudaError_t launch_preprocess_backward(const SceneView &s, const CamView &c, const uint32_t *tiles,
                                       const uint32_t *vis_index, const Ctl *ctl, const float4 *rec_grad,
                                       uint32_t grad_layer_mask, const gs_grads &g, float *contrib_sum,
                                       cudaStream_t st);

int sort_blocks();   // blocks of the sort / scan kernels on this device

// A positive value computed once per device ordinal (SM counts, occupancy and
// kernel attributes are properties of a device), safe to use from several
// host threads.  Ordinals beyond the table are computed on every call.
class PerDevice {
public:
    template <class F>
    int get(F compute) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return compute();
        std::lock_guard<std::mutex> lock(mu_);
        if (v_[dev] <= 0) v_[dev] = compute();
        return v_[dev];
    }

private:
    static constexpr int kDevices = 64;
    std::mutex mu_;
    int v_[kDevices] = {};
};
int report(int code, const char *msg);   // sets gs_last_error_string(), returns code

// Depth sort (sort.cu).  Buffers in the workspace:
struct SortWork {
    uint32_t *keys[2], *vals[2];   // ping-pong (key, Gaussian) buffers of the digit kernels, N each
    uint32_t *order;               // out: visible Gaussians in (depth, index) order, N
    uint32_t *vis_index;           // out: visible Gaussians in index order, N
    uint32_t *ghist;               // 4 x 256 digit histograms
    uint32_t *cnt;                 // sort_count_bytes(N): per-tile counts of the first digit
    uint32_t *grp;                 // sort_group_bytes(N): their sums per group of tiles
    uint64_t *status;              // sort_status_bytes(N): look-back words of the later digit kernels
};
uint32_t sort_tiles(int64_t n);
size_t sort_count_bytes(int64_t n);
size_t sort_group_bytes(int64_t n);
size_t sort_status_bytes(int64_t n);
// Sorts the Gaussians i < n with tiles[i] > 0 by (depth[i], i).  Histograms:
// the visible count (to ctl->n_vis and ctl->st.n_visible), the key range
// (ctl->depth_mm), the digit histograms and the per-tile counts of the
// first digit; these control words (with the tickets), work.ghist and
// work.grp must be zero on entry.  Digits: writes work.order and work.vis_index.
cudaError_t launch_sort_histograms(const uint32_t *tiles, const uint32_t *depth, int n, const SortWork &work,
                                   Ctl *ctl, cudaStream_t st);
cudaError_t launch_sort_digits(const uint32_t *tiles, const uint32_t *depth, int n, const SortWork &work, Ctl *ctl,
                               cudaStream_t st);
// Two eyes: Gaussians visible to view a or view b, keyed by depth_a where
// view a sees the Gaussian, else by depth_b (one depth order for both eyes).
cudaError_t launch_sort_histograms2(const uint32_t *tiles_a, const uint32_t *depth_a, const uint32_t *tiles_b,
                                    const uint32_t *depth_b, int n, const SortWork &work, Ctl *ctl, cudaStream_t st);
cudaError_t launch_sort_digits2(const uint32_t *tiles_a, const uint32_t *depth_a, const uint32_t *tiles_b,
                                const uint32_t *depth_b, int n, const SortWork &work, Ctl *ctl, cudaStream_t st);
// Tile binning (bin.cu).  Rows: splits the depth-ordered visible Gaussians
// (order[p], p < min(ctl->n_vis, n_cap)) into per-tile-row lists of
// (Gaussian, x0 | x1 << 16) in depth order; writes n_dup and the overflow
// status (n_dup > cap).  M: 2 kBinChunks Ty words; rows_buf: bin_rows_bytes(Ty),
// zero on entry.
cudaError_t launch_bin_rows(const uint32_t *order, const Rec *rec, uint32_t n_cap, int Ty, uint32_t *M,
                            void *rows_buf, uint2 *rowlist, Ctl *ctl, uint64_t cap, uint32_t piece, cudaStream_t st);
// Tiles: splits every row list into its tiles; writes the final Gaussian list
// (tile order, depth order within a tile) and every tile's [start, end).
// Does nothing when the status holds an error.
// P: bin_piece_bytes(cap, Tx, Ty) bytes; piece = bin_piece_entries(cap, Tx).
cudaError_t launch_bin_tiles(const uint2 *rowlist, const void *rows_buf, int Tx, int Ty, uint32_t piece, uint32_t *P,
                             uint32_t *list, uint2 *ranges, const Ctl *ctl, cudaStream_t st);
size_t bin_rows_bytes(int Ty);
uint32_t bin_piece_entries(int64_t dup_cap, int Tx);
size_t bin_piece_bytes(int64_t dup_cap, int Tx, int Ty);
// Training-step kernels (train.cu).
size_t loss_workspace_bytes(int W, int H);
cudaError_t launch_image_loss(const float *X, const float *A, const float *Ct, const float *At, float3 bg, int W,
                              int H, float lam, float w_a, void *ws, float *loss, float *dX, float *dA,
                              cudaStream_t st);
cudaError_t launch_adam(float *const p[5], const float *const g[5], float *const m[5], float *const v[5],
                        const uint32_t width[5], int64_t n, const uint8_t *layer, uint32_t train_mask,
                        const float lr[5], float beta1, float beta2, float eps, int step, cudaStream_t st);
cudaError_t launch_gather_rows(const void *src, void *dst, int64_t row_bytes, const int32_t *idx, int64_t n,
                               cudaStream_t st);
cudaError_t launch_activity(const float *const m[3], const float *const v[3], int sh_coeffs, int64_t n,
                            const uint8_t *layer, uint32_t train_mask, const float lr[3], float beta1, float beta2,
                            float eps, int step, float *activity, cudaStream_t st);
cudaError_t launch_activity_prune(const float *activity, const uint8_t *layer, uint32_t train_mask, int n,
                                  float samples, float thr, uint8_t *keep, int32_t *keep_index, int64_t *n_keep,
                                  uint32_t *partials, cudaStream_t st);
// SH codebook (codebook.cu).
cudaError_t launch_kmeans_assign(const float *pts, int64_t n, int dim, int64_t stride, const float *cent, int k,
                                 uint32_t *assign, cudaStream_t st);
cudaError_t launch_kmeans_update(const float *pts, int64_t n, int dim, int64_t stride, const uint32_t *assign, int k,
                                 float *cent, float *scratch, cudaStream_t st);
cudaError_t launch_sh_encode(const float *sh, int64_t n, int K, const uint32_t *assign, const float *cent, int k,
                             float *dc, uint16_t *index, void *table, cudaStream_t st);
cudaError_t launch_prune(const float *contrib_max, int n, float thr, uint8_t *keep, int32_t *keep_index,
                         int64_t *n_keep, uint32_t *partials, cudaStream_t st);

// Scratch of the compositor kernels (all in the render workspace).
struct CompositeBufs {
    uint32_t *order;      // [Tn] forward tile order (heaviest first)
    uint32_t *qdone;      // [8 Tn] per 8x8 block, a 64-bit word where its two forward blocks meet (FwdJob::qdone)
    uint32_t *seg_base;   // [Tn] first checkpoint segment of each tile
    uint32_t *qwork;      // [4 Tn] longest blended prefix of each 8x8 block (stored by the forward)
    float4 *ckpt;         // [segments][256] per-pixel (T, colour sum) every kSeg positions
    uint2 *items;         // backward work items (tile, block << 24 | segment), written by the forward
    uint32_t *n_items;
    uint32_t *queue;      // work-queue counter (forward and backward reuse it in turn)
};
// One view for the forward compositor.  A batch of views is composited by
// one persistent launch whose work queue spans all their tiles.
constexpr int kMaxBatch = GS_MAX_BATCH;
struct FwdJob {
    const uint32_t *order;
    const uint2 *ranges;
    const uint32_t *list;
    const Rec *rec;
    float *image, *alpha, *t_final;
    uint32_t *n_contrib;
    const uint32_t *seg_base;
    float4 *ckpt;
    uint32_t *qwork;
    unsigned long long *n_blended;   // the view's status word: blended pairs
    const Ctl *ctl;                  // the view's control block (bounds checks of GS_DEBUG builds)
    uint32_t n;                      // Gaussians of the view's scene
    uint32_t n_segs;                 // checkpoint segments the workspace holds
    int W, H, Tx, Tn;
    float3 bg;
    uint32_t *queue;       // the view's work-queue counter (zeroed by its set-up)
    uint2 *items;          // the view's backward work items, appended as the forward finishes 8x8 blocks
    uint32_t *n_items;     // their count (zero at the start of the render)
    uint32_t *qdone;       // [8 Tn] per 8x8 block, (finished 8x4 blocks << 32 | longest prefix) as 64 bits (zeroed by the set-up)
};
// Per-view set-up before compositing: tile order, checkpoint bases, zeroed
// block work and queue.  The backward's set-up also zeroes the record-gradient
// rows of the visible Gaussians (vis_index, *n_vis of the n Gaussians).
cudaError_t launch_fwd_setup(const CompositeBufs &cb, const uint2 *ranges, int Tn, cudaStream_t st);
// Composites n <= kMaxBatch views with one persistent launch; every view's
// queue must have been zeroed on the stream (its launch_fwd_setup does).
// wide_ok: the launch may take a third CTA per SM when it covers many pixels
// (gs_render, gs_render_stereo); batched serving launches, which share the GPU
// with a companion stream, keep two.
cudaError_t launch_composite_forward(const FwdJob *jobs, int n, cudaStream_t st, bool wide_ok);
// Backward set-up: work items (tile order by longest blended prefix) and the
// zeroed record-gradient rows of the visible Gaussians.
cudaError_t launch_bwd_setup(const CompositeBufs &cb, int Tx, int Ty, float4 *rec_grad, const uint32_t *vis_index,
                             const uint32_t *n_vis, int n, cudaStream_t st);
cudaError_t launch_composite_backward(const CompositeBufs &cb, const uint2 *ranges, const uint32_t *list,
                                      const Rec *rec, int W, int H, int Tx, int Ty, float3 bg, const float *t_final,
                                      const uint32_t *n_contrib, const float *dL_dimage,
                                      const float *dL_dalpha, const uint8_t *layer, uint32_t grad_layer_mask,
                                      float4 *rec_grad, float *contrib_max, uint32_t n, const Ctl *ctl,
                                      cudaStream_t st);

}  // namespace gs
