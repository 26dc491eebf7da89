// C ABI of the rasterizer (declared in include/gs.h): argument checks,
// workspace carve-up and the launch sequence of each entry point.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gs_internal.cuh"

namespace gs {

static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

bool make_layout(int64_t n, int W, int H, int64_t dup_cap, Layout *L) {
    if (n < 0 || n > 0x7FFFFFFF || W <= 0 || H <= 0 || W > GS_MAX_IMAGE_DIM || H > GS_MAX_IMAGE_DIM || dup_cap < 0 ||
        dup_cap > 0xFFFFFFFFLL)
        return false;
    Layout o;
    o.n = n; o.dup_cap = dup_cap; o.W = W; o.H = H;
    o.Tx = (W + kTile - 1) / kTile; o.Ty = (H + kTile - 1) / kTile;
    o.Tn = o.Tx * o.Ty;
    const size_t N = static_cast<size_t>(n), D = static_cast<size_t>(dup_cap), P = static_cast<size_t>(W) * H;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
    // the control block, the depth-sort histograms and group counts, the binning's per-row counters and the
    // tile ranges are adjacent: one memset per render clears them all
    o.ctl = take(256);
    o.sort_hist = take(4 * 256 * 4);
    o.sort_grp = take(sort_group_bytes(n));
    o.bin_rows = take(bin_rows_bytes(o.Ty));
    o.ranges = take(static_cast<size_t>(o.Tn) * 8);
    o.rec = take(N * sizeof(Rec));
    o.tiles = take(N * 4);
    o.depth = take(N * 4);
    o.sort_k[0] = take(N * 4); o.sort_k[1] = take(N * 4);
    o.sort_v[0] = take(N * 4); o.sort_v[1] = take(N * 4);
    o.order = take(N * 4);
    o.vis_index = take(N * 4);
    o.sort_cnt = take(sort_count_bytes(n));
    o.sort_status = take(sort_status_bytes(n));
    o.bin_m = take(static_cast<size_t>(kBinChunks) * o.Ty * 8);   // entries and pairs per (row, chunk)
    o.bin_piece = bin_piece_entries(dup_cap, o.Tx);
    o.bin_p = take(bin_piece_bytes(dup_cap, o.Tx, o.Ty));
    o.t_final = take(P * 4);
    o.n_contrib = take(P * 4);
    o.partials = take(kMaxSortBlocks * 4);
    o.rec_grad = take(N * sizeof(Rec));
    o.tile_order = take(static_cast<size_t>(o.Tn) * 4);
    o.qdone = take(static_cast<size_t>(o.Tn) * 32);
    o.seg_base = take(static_cast<size_t>(o.Tn) * 4);
    o.qwork = take(static_cast<size_t>(o.Tn) * 16);
    const size_t segs = D / kSeg + static_cast<size_t>(o.Tn) + 1;   // >= sum over tiles of ceil(len / kSeg)
    o.ckpt = take(segs * kTilePix * sizeof(float4));
    o.items = take(4 * segs * sizeof(uint2));
    o.rowlist = take(D * 8);     // row entries <= pairs
    o.list = take(D * 4);
    o.total = off;
    *L = o;
    return true;
}

int64_t capacity_for(int64_t n, int W, int H, size_t ws_bytes) {
    // The layout size grows monotonically with the capacity: binary search the
    // largest capacity that fits, so a workspace of gs_render_workspace_size(C)
    // bytes always holds at least C pairs.
    Layout L;
    if (!make_layout(n, W, H, 0, &L) || ws_bytes < L.total) return -1;
    int64_t lo = 0, hi = 0xFFFFFFFFLL;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (make_layout(n, W, H, mid, &L) && L.total <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace gs

using namespace gs;

namespace {

thread_local std::string g_err;

// ---- stage timing (off by default) ----
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<int, size_t>> marks;   // (stage, index of its start event)
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
};
Profiler g_prof;
std::atomic<int64_t> g_launches{0};

// NVTX range names of the stages (shown by profilers that record NVTX; the
// calls cost next to nothing when no tool is attached).
const char *const kStageNames[GS_STAGE_COUNT] = {
    "gs preprocess", "gs depth histograms", "gs depth sort", "gs bin rows", "gs bin tiles",
    "gs compositor set-up", "gs composite", "gs composite backward", "gs preprocess backward", "gs prune",
    "gs image loss", "gs adam"};

struct Stage {
    int stage;
    cudaStream_t st;
    size_t idx = 0;
    Stage(int s, cudaStream_t stream, int kernels) : stage(s), st(stream) {
        g_launches += kernels;
        nvtxRangePushA(kStageNames[s]);
        if (!g_prof.on) return;
        idx = g_prof.used;
        cudaEventRecord(g_prof.get(), st);
        g_prof.get();
    }
    ~Stage() {
        nvtxRangePop();
        if (!g_prof.on) return;
        cudaEventRecord(g_prof.pool[idx + 1], st);
        g_prof.marks.emplace_back(stage, idx);
    }
};

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GS_OK;
    return fail(GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_scene(const gs_scene *s, SceneView *v) {
    if (!s) return fail(GS_ERR_INVALID, "scene is NULL");
    if (s->n < 0 || s->n > 0x7FFFFFFF) return fail(GS_ERR_INVALID, "scene n out of range: %lld", (long long)s->n);
    if (s->sh_degree < 0 || s->sh_degree > 3) return fail(GS_ERR_INVALID, "sh_degree must be 0..3");
    if (s->dtype_scale_rot != GS_DTYPE_F32 && s->dtype_scale_rot != GS_DTYPE_F16 && s->dtype_scale_rot != GS_DTYPE_BF16)
        return fail(GS_ERR_INVALID, "unknown dtype %d", s->dtype_scale_rot);
    if (s->dtype_sh != GS_DTYPE_F32 && s->dtype_sh != GS_DTYPE_F16 && s->dtype_sh != GS_DTYPE_BF16 &&
        s->dtype_sh != GS_DTYPE_SH_CODEBOOK)
        return fail(GS_ERR_INVALID, "unknown dtype %d", s->dtype_sh);
    const bool cb = s->dtype_sh == GS_DTYPE_SH_CODEBOOK;
    if (cb && (s->sh_degree < 1 || s->sh_table_rows < 1 || s->sh_table_rows > 65536))
        return fail(GS_ERR_INVALID, "codebook SH needs sh_degree >= 1 and 1..65536 table rows");
    if (cb && s->n > 0 && (!s->sh_index || !s->sh_table || !aligned(s->sh_index, 16) || !aligned(s->sh_table, 16)))
        return fail(GS_ERR_INVALID, "codebook index and table must be set and 16-byte aligned");
    if (s->n > 0) {
        const void *ptrs[6] = {s->means, s->log_scales, s->quats, s->opacity_logit, s->sh, s->layer};
        for (const void *p : ptrs)
            if (!p) return fail(GS_ERR_INVALID, "scene array is NULL");
        for (const void *p : ptrs)
            if (!aligned(p, 16)) return fail(GS_ERR_INVALID, "scene arrays must be 16-byte aligned");
    }
    v->means = static_cast<const float *>(s->means);
    v->log_scales = s->log_scales;
    v->quats = s->quats;
    v->opacity_logit = static_cast<const float *>(s->opacity_logit);
    v->sh = s->sh;
    v->layer = s->layer;
    v->n = static_cast<int>(s->n);
    v->sh_degree = s->sh_degree;
    v->dtype_sh = s->dtype_sh;
    v->dtype_sr = s->dtype_scale_rot;
    v->sh_index = cb ? s->sh_index : nullptr;
    v->sh_table = cb ? s->sh_table : nullptr;
    v->sh_table_rows = cb ? s->sh_table_rows : 0;
    return GS_OK;
}

int check_camera(const gs_camera *c, CamView *v) {
    if (!c) return fail(GS_ERR_INVALID, "camera is NULL");
    if (c->width <= 0 || c->height <= 0 || c->width > GS_MAX_IMAGE_DIM || c->height > GS_MAX_IMAGE_DIM)
        return fail(GS_ERR_INVALID, "image size %dx%d outside 1..%d", c->width, c->height, GS_MAX_IMAGE_DIM);
    if (!(c->fx > 0.f) || !(c->fy > 0.f)) return fail(GS_ERR_INVALID, "focal lengths must be > 0");
    std::memcpy(v->R, c->R, sizeof v->R);
    std::memcpy(v->t, c->t, sizeof v->t);
    v->fx = c->fx; v->fy = c->fy; v->cx = c->cx; v->cy = c->cy; v->znear = c->znear;
    v->W = c->width; v->H = c->height;
    v->Tx = (c->width + kTile - 1) / kTile;
    v->Ty = (c->height + kTile - 1) / kTile;
    return GS_OK;
}


CompositeBufs composite_bufs(void *ws, const Layout &L) {
    Ctl *ctl = at<Ctl>(ws, L.ctl);
    CompositeBufs cb;
    cb.order = at<uint32_t>(ws, L.tile_order);
    cb.qdone = at<uint32_t>(ws, L.qdone);
    cb.seg_base = at<uint32_t>(ws, L.seg_base);
    cb.qwork = at<uint32_t>(ws, L.qwork);
    cb.ckpt = at<float4>(ws, L.ckpt);
    cb.items = at<uint2>(ws, L.items);
    cb.n_items = &ctl->n_items;
    cb.queue = &ctl->fwd_queue;
    return cb;
}

int workspace_layout(const gs_scene *s, const CamView &cv, void *ws, size_t ws_bytes, Layout *L) {
    if (!ws) return fail(GS_ERR_INVALID, "workspace is NULL");
    if (!aligned(ws, 256)) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
    const int64_t cap = capacity_for(s->n, cv.W, cv.H, ws_bytes);
    if (cap < 0) return fail(GS_ERR_WORKSPACE, "workspace of %zu bytes is below the fixed part", ws_bytes);
    if (!make_layout(s->n, cv.W, cv.H, cap, L)) return fail(GS_ERR_INVALID, "layout failed");
    return GS_OK;
}

}  // namespace

namespace gs {
// Records a message for gs_last_error_string() from other translation units.
int report(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace gs

extern "C" {

const char *gs_last_error_string(void) { return g_err.c_str(); }

const char *gs_version(void) {
#ifdef GS_DEBUG
    return "gs-layered-gb300 0.2 (sm_103a, GS_DEBUG bounds checks)";
#else
    return "gs-layered-gb300 0.2 (sm_103a)";
#endif
}

int gs_debug_build(void) {
#ifdef GS_DEBUG
    return 1;
#else
    return 0;
#endif
}

int gs_get_settings(gs_settings *out) {
    if (!out) return fail(GS_ERR_INVALID, "out is NULL");
    out->tile = kTile;
    out->dilation = kDilation;
    out->alpha_max = kAlphaMax;
    out->alpha_min = kAlphaMin;
    out->t_min = kTMin;
    out->frustum_clamp = kFrustumClamp;
    out->radius_sigmas = kRadiusSigmas;
    out->eigen_floor = kEigenFloor;
    out->checkpoint_stride = static_cast<int32_t>(kSeg);
    out->max_sh_degree = 3;
    out->max_planes = GS_MAX_PLANES;
    out->max_image_dim = GS_MAX_IMAGE_DIM;
    out->max_batch = GS_MAX_BATCH;
    out->debug_build = gs_debug_build();
    return GS_OK;
}

int gs_debug_site(const void *workspace, uint32_t *site, void *stream) {
#ifdef GS_DEBUG
    if (!workspace || !site) return fail(GS_ERR_INVALID, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = cuda_check(cudaMemcpyAsync(site, &static_cast<const Ctl *>(workspace)->dbg_site, sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, st),
                        "debug site copy");
    if (rc != GS_OK) return rc;
    return cuda_check(cudaStreamSynchronize(st), "debug site sync");
#else
    (void)workspace;
    (void)site;
    (void)stream;
    return fail(GS_ERR_INVALID, "gs_debug_site: only in GS_DEBUG builds");
#endif
}

int gs_render_workspace_size(int64_t n, int32_t width, int32_t height, int64_t dup_capacity, size_t *bytes) {
    if (!bytes) return fail(GS_ERR_INVALID, "bytes is NULL");
    Layout L;
    if (!make_layout(n, width, height, dup_capacity, &L)) return fail(GS_ERR_INVALID, "bad workspace sizes");
    *bytes = L.total;
    return GS_OK;
}

}  // extern "C"

namespace {

// Validates one view, launches S1 (preprocess) and S2 (binning and sorts) and
// the compositor set-up on st, and describes the view in *job.
// One view of a render call between its phases.
struct FrontCtx {
    SceneView sv;
    CamView cv;
    Layout L;
    void *ws = nullptr;
    Ctl *ctl = nullptr;
    Rec *rec = nullptr;
    uint32_t *tiles = nullptr;
    uint32_t *depth = nullptr;
    float *image = nullptr, *alpha = nullptr;
    float bg[3] = {0.f, 0.f, 0.f};
};

// Phase 1: validation, status reset and S1 (preprocess).
int front_preprocess(const gs_scene *scene, const gs_camera *camera, uint32_t layer_mask,
                     const gs_clip_plane *planes, int32_t n_planes, const float *bg, void *workspace,
                     size_t ws_bytes, float *image, float *alpha, cudaStream_t st, FrontCtx *f) {
    int rc;
    if ((rc = check_scene(scene, &f->sv)) != GS_OK) return rc;
    if ((rc = check_camera(camera, &f->cv)) != GS_OK) return rc;
    if (n_planes < 0 || n_planes > GS_MAX_PLANES) return fail(GS_ERR_INVALID, "n_planes must be 0..%d", GS_MAX_PLANES);
    if (n_planes > 0 && !planes) return fail(GS_ERR_INVALID, "planes is NULL");
    if (!bg) return fail(GS_ERR_INVALID, "bg is NULL");
    if (!image) return fail(GS_ERR_INVALID, "image is NULL");
    if ((rc = workspace_layout(scene, f->cv, workspace, ws_bytes, &f->L)) != GS_OK) return rc;
    Planes pl;
    std::memset(&pl, 0, sizeof pl);
    pl.n = n_planes;
    for (int k = 0; k < n_planes; ++k) {
        pl.p[k] = make_float4(planes[k].n[0], planes[k].n[1], planes[k].n[2], planes[k].d);
        pl.bits[k] = planes[k].layer_bits;
    }
    const Layout &L = f->L;
    f->ws = workspace;
    f->ctl = at<Ctl>(workspace, L.ctl);
    f->rec = at<Rec>(workspace, L.rec);
    f->tiles = at<uint32_t>(workspace, L.tiles);
    f->depth = at<uint32_t>(workspace, L.depth);
    f->image = image;
    f->alpha = alpha;
    for (int c = 0; c < 3; ++c) f->bg[c] = bg[c];
    // the control block and what follows it: depth-sort histograms and group counts, binning row counters, tile
    // ranges (all empty if the binning overflows)
    if ((rc = cuda_check(cudaMemsetAsync(f->ctl, 0, L.ranges + static_cast<size_t>(L.Tn) * 8 - L.ctl, st),
                         "memset status")) != GS_OK)
        return rc;
    Stage sg(GS_STAGE_PREPROCESS, st, 1);
    return cuda_check(launch_preprocess(f->sv, f->cv, layer_mask, pl, f->rec, f->tiles, f->depth, f->ctl, st),
                      "preprocess");
}

// Phase 2: the depth sort of the visible Gaussians.  With `other`, a
// Gaussian visible to either view is kept and keyed by this view's depth when
// this view sees it, else by the other's (shared stereo order).  Returns the
// depth order (in this view's workspace).
SortWork sort_work(void *ws, const Layout &L) {
    SortWork w;
    for (int k = 0; k < 2; ++k) {
        w.keys[k] = at<uint32_t>(ws, L.sort_k[k]);
        w.vals[k] = at<uint32_t>(ws, L.sort_v[k]);
    }
    w.order = at<uint32_t>(ws, L.order);
    w.vis_index = at<uint32_t>(ws, L.vis_index);
    w.ghist = at<uint32_t>(ws, L.sort_hist);
    w.cnt = at<uint32_t>(ws, L.sort_cnt);
    w.grp = at<uint32_t>(ws, L.sort_grp);
    w.status = at<uint64_t>(ws, L.sort_status);
    return w;
}

int front_sort(FrontCtx &f, const FrontCtx *other, cudaStream_t st, uint32_t **order) {
    const SortWork w = sort_work(f.ws, f.L);
    int rc;
    {
        Stage sg(GS_STAGE_COMPACT, st, 1);
        rc = other ? cuda_check(launch_sort_histograms2(f.tiles, f.depth, other->tiles, other->depth, f.sv.n, w,
                                                        f.ctl, st),
                                "depth histograms (stereo)")
                   : cuda_check(launch_sort_histograms(f.tiles, f.depth, f.sv.n, w, f.ctl, st), "depth histograms");
        if (rc != GS_OK) return rc;
    }
    {
        Stage sg(GS_STAGE_DEPTH_SORT, st, 4);
        rc = other ? cuda_check(launch_sort_digits2(f.tiles, f.depth, other->tiles, other->depth, f.sv.n, w, f.ctl,
                                                    st),
                                "depth sort (stereo)")
                   : cuda_check(launch_sort_digits(f.tiles, f.depth, f.sv.n, w, f.ctl, st), "depth sort");
        if (rc != GS_OK) return rc;
    }
    *order = w.order;
    return GS_OK;
}

// Phase 3: binning in the given depth order (whose count is at n_vis), the
// compositor set-up, and the forward job of the view.
int front_bin(FrontCtx &f, const uint32_t *order, cudaStream_t st, FwdJob *job) {
    int rc;
    const Layout &L = f.L;
    void *ws = f.ws;
    const uint32_t n = static_cast<uint32_t>(f.sv.n);
    uint32_t *list = at<uint32_t>(ws, L.list);
    uint2 *rowlist = at<uint2>(ws, L.rowlist);
    uint2 *ranges = at<uint2>(ws, L.ranges);
    {
        Stage sg(GS_STAGE_BIN_ROWS, st, 3);
        if ((rc = cuda_check(launch_bin_rows(order, f.rec, n, f.cv.Ty, at<uint32_t>(ws, L.bin_m),
                                             at<void>(ws, L.bin_rows), rowlist, f.ctl, L.dup_cap, L.bin_piece, st),
                             "binning rows")) != GS_OK)
            return rc;
    }
    {
        Stage sg(GS_STAGE_BIN_TILES, st, 3);
        if ((rc = cuda_check(launch_bin_tiles(rowlist, at<void>(ws, L.bin_rows), f.cv.Tx, f.cv.Ty, L.bin_piece,
                                              at<uint32_t>(ws, L.bin_p), list, ranges, f.ctl, st),
                             "binning tiles")) != GS_OK)
            return rc;
    }
    const CompositeBufs cb = composite_bufs(ws, L);
    {
        Stage sg(GS_STAGE_COMPOSITE_SETUP, st, 1);
        if ((rc = cuda_check(launch_fwd_setup(cb, ranges, L.Tn, st), "compositor set-up")) != GS_OK) return rc;
    }
    job->order = cb.order;
    job->ranges = ranges;
    job->list = list;
    job->rec = f.rec;
    job->image = f.image;
    job->alpha = f.alpha;
    job->t_final = at<float>(ws, L.t_final);
    job->n_contrib = at<uint32_t>(ws, L.n_contrib);
    job->seg_base = cb.seg_base;
    job->ckpt = cb.ckpt;
    job->qwork = cb.qwork;
    job->n_blended = reinterpret_cast<unsigned long long *>(&f.ctl->st.n_blended);
    job->ctl = f.ctl;
    job->n = n;
    job->n_segs = static_cast<uint32_t>(L.dup_cap / kSeg + L.Tn + 1);
    job->W = f.cv.W;
    job->H = f.cv.H;
    job->Tx = f.cv.Tx;
    job->Tn = L.Tn;
    job->bg = make_float3(f.bg[0], f.bg[1], f.bg[2]);
    job->queue = cb.queue;
    job->items = cb.items;
    job->n_items = cb.n_items;
    job->qdone = cb.qdone;
    return GS_OK;
}

// Validates one view, launches S1 (preprocess) and S2 (sort and binning) and
// the compositor set-up, and fills the view's forward job.
int render_front(const gs_scene *scene, const gs_camera *camera, uint32_t layer_mask, const gs_clip_plane *planes,
                 int32_t n_planes, const float *bg, void *workspace, size_t ws_bytes, float *image, float *alpha,
                 cudaStream_t st, FwdJob *job) {
    FrontCtx f;
    int rc = front_preprocess(scene, camera, layer_mask, planes, n_planes, bg, workspace, ws_bytes, image, alpha, st,
                              &f);
    if (rc != GS_OK) return rc;
    uint32_t *order = nullptr;
    if ((rc = front_sort(f, nullptr, st, &order)) != GS_OK) return rc;
    return front_bin(f, order, st, job);
}

}  // namespace

extern "C" {

int gs_render(const gs_scene *scene, const gs_camera *camera, uint32_t layer_mask, const gs_clip_plane *planes,
              int32_t n_planes, const float *bg, void *workspace, size_t ws_bytes, float *image, float *alpha,
              void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FwdJob job;
    int rc = render_front(scene, camera, layer_mask, planes, n_planes, bg, workspace, ws_bytes, image, alpha, st, &job);
    if (rc != GS_OK) return rc;
    Stage sg(GS_STAGE_COMPOSITE, st, 1);
    return cuda_check(launch_composite_forward(&job, 1, st, true), "composite");
}

int gs_render_batch(const gs_render_request *reqs, int32_t n, void *stream) {
    if (!reqs || n < 1 || n > GS_MAX_BATCH) return fail(GS_ERR_INVALID, "n must be 1..%d", GS_MAX_BATCH);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j)
            if (reqs[i].workspace == reqs[j].workspace)
                return fail(GS_ERR_INVALID, "requests %d and %d share a workspace", j, i);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FwdJob jobs[GS_MAX_BATCH];
    for (int i = 0; i < n; ++i) {
        const gs_render_request &r = reqs[i];
        int rc = render_front(r.scene, r.camera, r.layer_mask, r.planes, r.n_planes, r.bg, r.workspace, r.ws_bytes,
                              r.image, r.alpha, st, &jobs[i]);
        if (rc != GS_OK) return rc;
    }
    Stage sg(GS_STAGE_COMPOSITE, st, 1);
    return cuda_check(launch_composite_forward(jobs, n, st, false), "batched composite");
}


int gs_render_stereo(const gs_scene *scene, const gs_camera *left, const gs_camera *right, uint32_t layer_mask,
                     const gs_clip_plane *planes, int32_t n_planes, const float *bg, void *ws_left,
                     size_t ws_left_bytes, void *ws_right, size_t ws_right_bytes, float *image_left,
                     float *alpha_left, float *image_right, float *alpha_right, int32_t shared_sort, void *stream) {
    if (ws_left == ws_right) return fail(GS_ERR_INVALID, "the two eyes need separate workspaces");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FrontCtx f[2];
    int rc;
    if ((rc = front_preprocess(scene, left, layer_mask, planes, n_planes, bg, ws_left, ws_left_bytes, image_left,
                               alpha_left, st, &f[0])) != GS_OK)
        return rc;
    if ((rc = front_preprocess(scene, right, layer_mask, planes, n_planes, bg, ws_right, ws_right_bytes, image_right,
                               alpha_right, st, &f[1])) != GS_OK)
        return rc;
    FwdJob jobs[2];
    if (shared_sort) {
        uint32_t *order = nullptr;
        if ((rc = front_sort(f[0], &f[1], st, &order)) != GS_OK) return rc;
        // the right eye bins in the shared order: it needs the shared count, and
        // its backward the visible list, too
        if ((rc = cuda_check(cudaMemcpyAsync(at<uint32_t>(f[1].ws, f[1].L.vis_index),
                                             at<uint32_t>(f[0].ws, f[0].L.vis_index),
                                             static_cast<size_t>(f[0].sv.n) * sizeof(uint32_t),
                                             cudaMemcpyDeviceToDevice, st),
                             "shared visible list")) != GS_OK)
            return rc;
        if ((rc = cuda_check(cudaMemcpyAsync(&f[1].ctl->n_vis, &f[0].ctl->n_vis, sizeof(uint32_t),
                                             cudaMemcpyDeviceToDevice, st),
                             "shared count")) != GS_OK)
            return rc;
        if ((rc = cuda_check(cudaMemcpyAsync(&f[1].ctl->st.n_visible, &f[0].ctl->st.n_visible, sizeof(uint32_t),
                                             cudaMemcpyDeviceToDevice, st),
                             "shared count")) != GS_OK)
            return rc;
        if ((rc = front_bin(f[0], order, st, &jobs[0])) != GS_OK) return rc;
        if ((rc = front_bin(f[1], order, st, &jobs[1])) != GS_OK) return rc;
    } else {
        for (int e = 0; e < 2; ++e) {
            uint32_t *order = nullptr;
            if ((rc = front_sort(f[e], nullptr, st, &order)) != GS_OK) return rc;
            if ((rc = front_bin(f[e], order, st, &jobs[e])) != GS_OK) return rc;
        }
    }
    Stage sg(GS_STAGE_COMPOSITE, st, 1);
    return cuda_check(launch_composite_forward(jobs, 2, st, true), "stereo composite");
}

int gs_render_backward(const gs_scene *scene, const gs_camera *camera, const float *bg, void *workspace,
                       size_t ws_bytes, const float *dL_dimage, const float *dL_dalpha, uint32_t grad_layer_mask,
                       const gs_grads *grads, float *contrib_sum, float *contrib_max, void *stream) {
    SceneView sv;
    CamView cv;
    int rc;
    if ((rc = check_scene(scene, &sv)) != GS_OK) return rc;
    if ((rc = check_camera(camera, &cv)) != GS_OK) return rc;
    if (sv.dtype_sh == GS_DTYPE_SH_CODEBOOK) return fail(GS_ERR_INVALID, "codebook SH is render only");
    if (!bg) return fail(GS_ERR_INVALID, "bg is NULL");
    if (!grads || (sv.n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logit ||
                                !grads->sh)))
        return fail(GS_ERR_INVALID, "gradient outputs must all be set");
    Layout L;
    if ((rc = workspace_layout(scene, cv, workspace, ws_bytes, &L)) != GS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *ws = workspace;
    float4 *rec_grad = at<float4>(ws, L.rec_grad);
    {
        Stage sg(GS_STAGE_COMPOSITE_SETUP, st, 1);     // with the record-gradient zeroing
        if ((rc = cuda_check(launch_bwd_setup(composite_bufs(ws, L), cv.Tx, cv.Ty, rec_grad,
                                              at<uint32_t>(ws, L.vis_index), &at<Ctl>(ws, L.ctl)->n_vis, sv.n, st),
                             "backward set-up")) != GS_OK)
            return rc;
    }
    {
        Stage sg(GS_STAGE_COMPOSITE_BWD, st, 1);
        if ((rc = cuda_check(launch_composite_backward(composite_bufs(ws, L), at<uint2>(ws, L.ranges),
                                                       at<uint32_t>(ws, L.list), at<Rec>(ws, L.rec), cv.W, cv.H,
                                                       cv.Tx, cv.Ty, make_float3(bg[0], bg[1], bg[2]),
                                                       at<float>(ws, L.t_final), at<uint32_t>(ws, L.n_contrib),
                                                       dL_dimage, dL_dalpha, sv.layer, grad_layer_mask, rec_grad,
                                                       contrib_max, static_cast<uint32_t>(sv.n), at<Ctl>(ws, L.ctl),
                                                       st),
                             "composite backward")) != GS_OK)
            return rc;
    }
    Stage sg(GS_STAGE_PREPROCESS_BWD, st, 1);
    return cuda_check(launch_preprocess_backward(sv, cv, at<uint32_t>(ws, L.tiles), at<uint32_t>(ws, L.vis_index),
                                                 at<Ctl>(ws, L.ctl), rec_grad, grad_layer_mask, *grads, contrib_sum,
                                                 st),
                      "preprocess backward");
}

int gs_workspace_layout(int64_t n, int32_t width, int32_t height, size_t ws_bytes, int64_t *out) {
    if (!out) return fail(GS_ERR_INVALID, "out is NULL");
    const int64_t cap = capacity_for(n, width, height, ws_bytes);
    if (cap < 0) return fail(GS_ERR_WORKSPACE, "workspace of %zu bytes is below the fixed part", ws_bytes);
    Layout L;
    if (!make_layout(n, width, height, cap, &L)) return fail(GS_ERR_INVALID, "bad sizes");
    const int64_t v[GS_LAYOUT_COUNT] = {
        (int64_t)L.ctl, (int64_t)L.rec, (int64_t)L.tiles, (int64_t)L.depth, (int64_t)L.list, (int64_t)L.ranges, (int64_t)L.t_final, (int64_t)L.n_contrib,
        (int64_t)L.rec_grad, (int64_t)L.total, cap};
    for (int k = 0; k < GS_LAYOUT_COUNT; ++k) out[k] = v[k];
    return GS_OK;
}

int gs_prune_workspace_size(int64_t n, size_t *bytes) {
    if (!bytes) return fail(GS_ERR_INVALID, "bytes is NULL");
    if (n < 0 || n > 0x7FFFFFFF) return fail(GS_ERR_INVALID, "n out of range");
    *bytes = kMaxSortBlocks * 4 + sizeof(Ctl);
    return GS_OK;
}

int gs_contrib_prune(const float *contrib_max, int64_t n, float threshold, uint8_t *keep, int32_t *keep_index,
                     int64_t *n_keep, void *workspace, size_t ws_bytes, void *stream) {
    if (n < 0 || n > 0x7FFFFFFF) return fail(GS_ERR_INVALID, "n out of range");
    if (!n_keep) return fail(GS_ERR_INVALID, "n_keep is NULL");
    if (n > 0 && (!contrib_max || !keep)) return fail(GS_ERR_INVALID, "contrib_max and keep must be set");
    size_t need = 0;
    gs_prune_workspace_size(n, &need);
    if (!workspace || ws_bytes < need) return fail(GS_ERR_WORKSPACE, "prune workspace needs %zu bytes", need);
    if (!aligned(workspace, 16)) return fail(GS_ERR_INVALID, "workspace must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Stage sg(GS_STAGE_PRUNE, st, 2);
    return cuda_check(launch_prune(contrib_max, static_cast<int>(n), threshold, keep, keep_index, n_keep,
                                   static_cast<uint32_t *>(workspace), st),
                      "prune");
}

int gs_profile_enable(int on) {
    g_prof.on = on != 0;
    return GS_OK;
}

int gs_profile_collect(double *ms, int64_t *calls) {
    if (!ms || !calls) return fail(GS_ERR_INVALID, "NULL argument");
    for (int k = 0; k < GS_STAGE_COUNT; ++k) { ms[k] = 0.0; calls[k] = 0; }
    for (auto &m : g_prof.marks) {
        cudaEvent_t b = g_prof.pool[m.second], e = g_prof.pool[m.second + 1];
        int rc = cuda_check(cudaEventSynchronize(e), "profile sync");
        if (rc != GS_OK) return rc;
        float t = 0.f;
        if ((rc = cuda_check(cudaEventElapsedTime(&t, b, e), "profile elapsed")) != GS_OK) return rc;
        ms[m.first] += t;
        calls[m.first] += 1;
    }
    g_prof.marks.clear();
    g_prof.used = 0;
    return GS_OK;
}

int64_t gs_kernel_launches(void) { return g_launches.load(); }

int gs_image_loss_workspace_size(int32_t width, int32_t height, size_t *bytes) {
    if (!bytes) return fail(GS_ERR_INVALID, "bytes is NULL");
    if (width <= 0 || height <= 0 || width > GS_MAX_IMAGE_DIM || height > GS_MAX_IMAGE_DIM)
        return fail(GS_ERR_INVALID, "image size %dx%d outside 1..%d", width, height, GS_MAX_IMAGE_DIM);
    *bytes = loss_workspace_bytes(width, height);
    return GS_OK;
}

int gs_image_loss(const float *image, const float *alpha, const float *target_rgb, const float *target_alpha,
                  const float *bg, int32_t width, int32_t height, float lambda_dssim, float w_alpha,
                  void *workspace, size_t ws_bytes, float *loss, float *dL_dimage, float *dL_dalpha,
                  void *stream) {
    size_t need = 0;
    int rc = gs_image_loss_workspace_size(width, height, &need);
    if (rc != GS_OK) return rc;
    if (!image || !target_rgb || !target_alpha || !bg || !loss || !dL_dimage || !workspace)
        return fail(GS_ERR_INVALID, "NULL argument");
    if (ws_bytes < need) return fail(GS_ERR_WORKSPACE, "loss workspace of %zu bytes, need %zu", ws_bytes, need);
    if (!aligned(workspace, 256)) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
    if (!(lambda_dssim >= 0.f && lambda_dssim <= 1.f) || !(w_alpha >= 0.f))
        return fail(GS_ERR_INVALID, "lambda_dssim must be in [0, 1] and w_alpha >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!alpha && dL_dalpha &&
        (rc = cuda_check(cudaMemsetAsync(dL_dalpha, 0, static_cast<size_t>(width) * height * 4, st),
                         "zero dL_dalpha")) != GS_OK)
        return rc;
    Stage sg(GS_STAGE_LOSS, st, 3);
    return cuda_check(launch_image_loss(image, alpha, target_rgb, target_alpha, make_float3(bg[0], bg[1], bg[2]),
                                        width, height, lambda_dssim, w_alpha, workspace, loss, dL_dimage,
                                        alpha ? dL_dalpha : nullptr, st),
                      "image loss");
}

int gs_adam_step(const gs_scene *scene, const gs_grads *grads, const gs_adam_state *state, const float *lr,
                 float beta1, float beta2, float eps, int32_t step, uint32_t train_layer_mask, void *stream) {
    SceneView sv;
    int rc;
    if ((rc = check_scene(scene, &sv)) != GS_OK) return rc;
    if (!grads || !state || !lr) return fail(GS_ERR_INVALID, "NULL argument");
    if (sv.dtype_sh != GS_DTYPE_F32 || sv.dtype_sr != GS_DTYPE_F32)
        return fail(GS_ERR_INVALID, "Adam updates float32 parameters only");
    if (step < 1) return fail(GS_ERR_INVALID, "step must be >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
        return fail(GS_ERR_INVALID, "bad Adam hyper-parameters");
    if (sv.n == 0) return GS_OK;
    const int K = (sv.sh_degree + 1) * (sv.sh_degree + 1);
    float *p[5] = {const_cast<float *>(sv.means), static_cast<float *>(const_cast<void *>(sv.log_scales)),
                   static_cast<float *>(const_cast<void *>(sv.quats)), const_cast<float *>(sv.opacity_logit),
                   static_cast<float *>(const_cast<void *>(sv.sh))};
    const float *g[5] = {grads->means, grads->log_scales, grads->quats, grads->opacity_logit, grads->sh};
    const uint32_t width[5] = {3, 3, 4, 1, static_cast<uint32_t>(3 * K)};
    for (int k = 0; k < 5; ++k)
        if (!g[k] || !state->m[k] || !state->v[k]) return fail(GS_ERR_INVALID, "gradient or moment array is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Stage sg(GS_STAGE_ADAM, st, 1);
    return cuda_check(launch_adam(p, g, state->m, state->v, width, sv.n, sv.layer, train_layer_mask, lr, beta1, beta2,
                                  eps, step, st),
                      "adam");
}

int gs_activity_accumulate(const gs_adam_state *state, const uint8_t *layer, int64_t n, int32_t sh_degree,
                           const float *lr, float beta1, float beta2, float eps, int32_t step,
                           uint32_t train_layer_mask, float *activity, void *stream) {
    if (n < 0 || n > 0x7FFFFFFF) return fail(GS_ERR_INVALID, "n out of range");
    if (sh_degree < 0 || sh_degree > 3) return fail(GS_ERR_INVALID, "sh_degree must be 0..3");
    if (step < 1) return fail(GS_ERR_INVALID, "step must be >= 1");
    if (!state || !lr) return fail(GS_ERR_INVALID, "NULL argument");
    if (n == 0) return GS_OK;
    if (!layer || !activity || !state->m[0] || !state->v[0] || !state->m[1] || !state->v[1] || !state->m[4] ||
        !state->v[4])
        return fail(GS_ERR_INVALID, "NULL array");
    const float *m[3] = {state->m[0], state->m[4], state->m[1]};
    const float *v[3] = {state->v[0], state->v[4], state->v[1]};
    const float l3[3] = {lr[0], lr[4], lr[1]};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Stage sg(GS_STAGE_ADAM, st, 1);
    return cuda_check(launch_activity(m, v, (sh_degree + 1) * (sh_degree + 1), n, layer, train_layer_mask, l3, beta1,
                                      beta2, eps, step, activity, st),
                      "activity");
}

int gs_activity_prune(const float *activity, const uint8_t *layer, int64_t n, uint32_t train_layer_mask,
                      float samples, float threshold, uint8_t *keep, int32_t *keep_index, int64_t *n_keep,
                      void *workspace, size_t ws_bytes, void *stream) {
    if (n < 0 || n > 0x7FFFFFFF) return fail(GS_ERR_INVALID, "n out of range");
    if (!n_keep) return fail(GS_ERR_INVALID, "n_keep is NULL");
    if (n > 0 && (!activity || !layer || !keep)) return fail(GS_ERR_INVALID, "activity, layer and keep must be set");
    if (!(samples > 0.f)) return fail(GS_ERR_INVALID, "samples must be > 0");
    size_t need = 0;
    gs_prune_workspace_size(n, &need);
    if (!workspace || ws_bytes < need) return fail(GS_ERR_WORKSPACE, "prune workspace needs %zu bytes", need);
    if (!aligned(workspace, 16)) return fail(GS_ERR_INVALID, "workspace must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Stage sg(GS_STAGE_PRUNE, st, 2);
    return cuda_check(launch_activity_prune(activity, layer, train_layer_mask, static_cast<int>(n), samples, threshold,
                                            keep, keep_index, n_keep, static_cast<uint32_t *>(workspace), st),
                      "activity prune");
}

int gs_kmeans_scratch_size(int32_t k, int32_t dim, size_t *bytes) {
    if (!bytes) return fail(GS_ERR_INVALID, "bytes is NULL");
    if (k < 1 || dim < 1 || dim > kCbMaxDim) return fail(GS_ERR_INVALID, "k >= 1 and 1 <= dim <= %d", kCbMaxDim);
    *bytes = static_cast<size_t>(k) * (dim + 1) * sizeof(float);
    return GS_OK;
}

int gs_kmeans_assign(const float *points, int64_t n, int32_t dim, int64_t stride, const float *centroids, int32_t k,
                     uint32_t *assign, void *stream) {
    if (n < 0 || k < 1 || dim < 1 || dim > kCbMaxDim || stride < dim)
        return fail(GS_ERR_INVALID, "bad sizes (n %lld, k %d, dim %d, stride %lld)", (long long)n, k, dim,
                    (long long)stride);
    if (n > 0 && (!points || !centroids || !assign)) return fail(GS_ERR_INVALID, "NULL argument");
    return cuda_check(launch_kmeans_assign(points, n, dim, stride, centroids, k, assign,
                                           static_cast<cudaStream_t>(stream)),
                      "kmeans assign");
}

int gs_kmeans_update(const float *points, int64_t n, int32_t dim, int64_t stride, const uint32_t *assign, int32_t k,
                     float *centroids, void *scratch, size_t scratch_bytes, void *stream) {
    size_t need = 0;
    int rc = gs_kmeans_scratch_size(k, dim, &need);
    if (rc != GS_OK) return rc;
    if (n < 0 || stride < dim) return fail(GS_ERR_INVALID, "bad sizes");
    if (!centroids || !scratch || (n > 0 && (!points || !assign))) return fail(GS_ERR_INVALID, "NULL argument");
    if (scratch_bytes < need) return fail(GS_ERR_WORKSPACE, "k-means scratch needs %zu bytes", need);
    return cuda_check(launch_kmeans_update(points, n, dim, stride, assign, k, centroids, static_cast<float *>(scratch),
                                           static_cast<cudaStream_t>(stream)),
                      "kmeans update");
}

int gs_sh_codebook_encode(const float *sh, int64_t n, int32_t sh_degree, const uint32_t *assign,
                          const float *centroids, int32_t k, float *dc, uint16_t *index, void *table, void *stream) {
    if (n < 0 || sh_degree < 1 || sh_degree > 3 || k < 1 || k > 65536)
        return fail(GS_ERR_INVALID, "bad sizes (n %lld, degree %d, k %d)", (long long)n, sh_degree, k);
    if (!centroids || !table || (n > 0 && (!sh || !assign || !dc || !index))) return fail(GS_ERR_INVALID, "NULL argument");
    const int K = (sh_degree + 1) * (sh_degree + 1);
    return cuda_check(launch_sh_encode(sh, n, K, assign, centroids, k, dc, index, table,
                                       static_cast<cudaStream_t>(stream)),
                      "sh codebook encode");
}

int gs_gather_rows(const void *src, void *dst, int64_t row_bytes, const int32_t *index, int64_t n, void *stream) {
    if (n < 0 || row_bytes <= 0 || row_bytes > 0x7FFFFFFF) return fail(GS_ERR_INVALID, "bad row size or count");
    if (n > 0 && (!src || !dst || !index)) return fail(GS_ERR_INVALID, "NULL argument");
    if ((row_bytes % 2 == 0) && (!aligned(src, 2) || !aligned(dst, 2)))
        return fail(GS_ERR_INVALID, "rows of an even byte count must be 2-byte aligned");
    return cuda_check(launch_gather_rows(src, dst, row_bytes, index, n, static_cast<cudaStream_t>(stream)),
                      "gather rows");
}

int gs_read_status(const void *workspace, gs_status *out, void *stream) {
    if (!workspace || !out) return fail(GS_ERR_INVALID, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = cuda_check(cudaMemcpyAsync(out, workspace, sizeof(gs_status), cudaMemcpyDeviceToHost, st), "status copy");
    if (rc != GS_OK) return rc;
    return cuda_check(cudaStreamSynchronize(st), "status sync");
}

}  // extern "C"
