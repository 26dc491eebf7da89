/*
 * gs.h - C ABI of the layered Gaussian-splatting tile rasterizer (GB300, sm_103a).
 *
 * Paper: "Multi-Layer Gaussian Splatting for Immersive Anatomy Visualization".
 * The scene is one Gaussian cloud whose points carry a layer id stored next to
 * their colour and scale attributes (Sec. 3.2).  Layers are rendered alone or
 * together and can be cut (Sec. 1, Sec. 3.3, Sec. 5); the renderer sorts the
 * Gaussians relative to the camera and splats them (Sec. 3.3) following the
 * EWA / 3DGS formulation the paper cites (Sec. 2.2.1); training a layer needs
 * the gradient of that render with the lower layers frozen (Sec. 3.2) and the
 * per-Gaussian contribution used to remove inactive Gaussians (Sec. 3.2.2).
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller, unless the
 *     comment says "host".  The library never allocates device memory on these
 *     paths and never frees what it is given.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and never synchronise, except gs_read_status.
 *   - Every call returns GS_OK or an error code; gs_last_error_string() gives a
 *     message for the calling thread's last failure.  Argument errors are
 *     detected on the host before any launch (GS_ERR_INVALID).  Errors that can
 *     only be known on the device (duplicate-list overflow) are written to the
 *     status word at the start of the workspace; read it with gs_read_status.
 *   - Images are planar float32: image[c][y][x], c in {R,G,B}; per-pixel
 *     arrays are [y][x].  Pixel (x, y) is sampled at (x + 0.5, y + 0.5).
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GS_OK = 0,
    GS_ERR_INVALID = 1,    /* bad argument (null pointer, size, dtype, ...) */
    GS_ERR_WORKSPACE = 2,  /* workspace too small (host check) or duplicate-list overflow (device status) */
    GS_ERR_CUDA = 3,       /* a CUDA runtime call or launch failed */
    GS_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up */
    GS_ERR_OOM = 5,        /* an admission/memory budget was exceeded */
    GS_ERR_BOUNDS = 6      /* a bounds check of a GS_DEBUG build failed (device status; the access was skipped) */
};

enum { GS_DTYPE_F32 = 0, GS_DTYPE_F16 = 1, GS_DTYPE_BF16 = 2, GS_DTYPE_SH_CODEBOOK = 3 };

#define GS_TILE 16          /* tile edge in pixels */
#define GS_MAX_PLANES 8     /* clip planes per call */
#define GS_MAX_IMAGE_DIM 4096   /* largest image width and height */
#define GS_MAX_LAYERS 32    /* layer ids 0..31 (bit L of a mask = layer L) */

/* Pinhole camera, world -> camera p = R mu + t, OpenCV axes (x right, y down,
 * z forward).  R is row-major.  fx, fy, cx, cy in pixels; width and height
 * in 1..GS_MAX_IMAGE_DIM (GS_ERR_INVALID otherwise); Gaussians with
 * p_z <= znear are culled (0.2 in every workload here).                       */
typedef struct gs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    float _reserved;
} gs_camera;

/* Clip plane (cutting, Sec. 5): a Gaussian whose layer bit is set in
 * layer_bits is removed whole when n . mu + d < 0 (its centre is tested).     */
typedef struct gs_clip_plane {
    float n[3];
    float d;
    uint32_t layer_bits;
    uint32_t _reserved;
} gs_clip_plane;

/* Layered Gaussian scene (device pointers, read only), N Gaussians:
 *   means          float32 [N][3]
 *   log_scales     [N][3]  dtype_scale_rot (f32 / f16 / bf16)
 *   quats          [N][4]  dtype_scale_rot, (w, x, y, z), need not be unit
 *   opacity_logit  float32 [N]              opacity = sigmoid(logit)
 *   sh             [N][K][3] dtype_sh, K = (sh_degree+1)^2, real SH with the
 *                  Condon-Shortley phase, index k = l*l + l + m
 *   layer          uint8 [N], values 0..31
 * With dtype_sh = GS_DTYPE_SH_CODEBOOK (Sec. 3.3: K-means clustering of the
 * SH coefficients; render only, sh_degree >= 1): sh is the DC coefficient
 * float32 [N][3]; sh_index uint16 [N] selects a row of sh_table, FP16
 * [sh_table_rows][R] with R = 3(K-1) rounded up to a multiple of 8 (the
 * coefficients k = 1..K-1, channel fastest, then zero padding).  Both fields
 * are ignored for the other dtypes.  Every pointer must be 16-byte aligned. */
typedef struct gs_scene {
    const void *means;
    const void *log_scales;
    const void *quats;
    const void *opacity_logit;
    const void *sh;
    const uint8_t *layer;
    int64_t n;
    int32_t sh_degree;      /* 0..3 */
    int32_t dtype_sh;       /* GS_DTYPE_* */
    int32_t dtype_scale_rot;/* GS_DTYPE_F32 / F16 / BF16 */
    int32_t sh_table_rows;  /* codebook rows (1..65536), GS_DTYPE_SH_CODEBOOK only */
    const uint16_t *sh_index;
    const void *sh_table;
} gs_scene;

/* Gradient outputs (device, float32, same shapes as the scene fields).  Every
 * element is written (overwritten, not accumulated); Gaussians that were not
 * rendered or whose layer is not in grad_layer_mask receive 0.               */
typedef struct gs_grads {
    float *means;           /* [N][3] */
    float *log_scales;      /* [N][3] */
    float *quats;           /* [N][4] */
    float *opacity_logit;   /* [N]    */
    float *sh;              /* [N][K][3] */
} gs_grads;

/* Device status word at offset 0 of a render workspace. */
typedef struct gs_status {
    int32_t error;          /* GS_OK, or GS_ERR_WORKSPACE when n_dup > dup_capacity */
    uint32_t n_visible;     /* Gaussians that survived every cull */
    uint64_t n_dup;         /* (tile, Gaussian) pairs the frame needs */
    uint64_t dup_capacity;  /* pairs the workspace can hold */
    uint64_t n_blended;     /* (pixel, Gaussian) pairs blended by the last forward composite */
} gs_status;

/* Bytes of workspace for rendering n Gaussians at width x height with room for
 * dup_capacity (tile, Gaussian) pairs (each visible Gaussian needs one pair per
 * tile its 3-sigma square touches).  The workspace also keeps the forward state
 * that gs_render_backward reads.  Returns GS_ERR_INVALID on bad sizes.       */
int gs_render_workspace_size(int64_t n, int32_t width, int32_t height, int64_t dup_capacity,
                             size_t *bytes);

/* Forward render (steps: preprocess -> depth sort -> tile binning -> tile
 * sort -> front-to-back compositing), Sec. 3.3.
 *   layer_mask  bit L renders layer L (Sec. 3.3: only active layers)
 *   planes      HOST array of n_planes clip planes (0 <= n_planes <= 8)
 *   bg          HOST float[3] background colour
 *   workspace   device buffer of ws_bytes (>= gs_render_workspace_size for
 *               some capacity); 256-byte aligned; keeps the forward state
 *   image       [3][H][W] = sum_i c_i a_i T_i + T_final * bg
 *   alpha       [H][W] = 1 - T_final (may be NULL)
 * If the frame needs more pairs than the workspace holds, the status word
 * reports GS_ERR_WORKSPACE and the required n_dup; the image is then
 * incomplete (never out of bounds).                                          */
int gs_render(const gs_scene *scene, const gs_camera *camera, uint32_t layer_mask,
              const gs_clip_plane *planes, int32_t n_planes, const float *bg,
              void *workspace, size_t ws_bytes, float *image, float *alpha, void *stream);

/* Several views rendered as one batch (serving; stereo eyes).  Equivalent to
 * gs_render for each request in order on `stream` (each with its own
 * workspace, image and alpha), except that the compositing of all views is
 * one persistent launch whose work queue spans every view's tiles, so small
 * views share the GPU instead of each leaving most of it idle.  1 <= n <=
 * GS_MAX_BATCH; workspaces must be distinct (GS_ERR_INVALID otherwise).
 * Each workspace afterwards holds its view's forward state, so
 * gs_render_backward can be called per view.                                */
#define GS_MAX_BATCH 16
typedef struct gs_render_request {
    const gs_scene *scene;
    const gs_camera *camera;
    uint32_t layer_mask;
    int32_t n_planes;
    const gs_clip_plane *planes;    /* host array */
    float bg[3];                    /* host values */
    float _reserved;
    void *workspace;
    size_t ws_bytes;
    float *image;
    float *alpha;                   /* may be NULL */
} gs_render_request;
int gs_render_batch(const gs_render_request *reqs, int32_t n, void *stream);

/* Stereo pair (Sec. 3.3: a VR frame renders the scene once per eye) of one
 * scene with the same layer mask and clip planes: each eye as gs_render on
 * its own workspace, both eyes composited by one launch.  shared_sort != 0
 * sorts once for both eyes, as the paper's renderer can: the Gaussians
 * visible to either eye are ordered by their depth in the left eye (by the
 * right eye's depth when only the right eye sees them), and both eyes bin
 * and composite in that order.  The left image is then exactly gs_render's;
 * the right image differs only where splats change depth order between the
 * eyes (an approximation).  With shared_sort, the left status word's
 * n_visible counts the Gaussians visible to either eye.  Workspaces must be
 * distinct; either eye's pair list may overflow independently (status word
 * of that workspace).                                                        */
int gs_render_stereo(const gs_scene *scene, const gs_camera *left, const gs_camera *right, uint32_t layer_mask,
                     const gs_clip_plane *planes, int32_t n_planes, const float *bg, void *ws_left,
                     size_t ws_left_bytes, void *ws_right, size_t ws_right_bytes, float *image_left,
                     float *alpha_left, float *image_right, float *alpha_right, int32_t shared_sort, void *stream);

/* Backward of the last gs_render made with this workspace (same scene, camera
 * and bg; Sec. 3.2 layered training).
 *   dL_dimage  [3][H][W], dL_dalpha [H][W] (either may be NULL = zero)
 *   grad_layer_mask  layers that receive gradients; others are frozen (Sec. 3.2)
 *   grads      outputs (see gs_grads)
 *   contrib_sum, contrib_max  [N] float32, ACCUMULATED across calls: += sum
 *              and max over blended pixels of alpha*T (Sec. 3.2.2).  Either
 *              may be NULL.  Zero them before the first view.
 * The library's scratch for per-Gaussian record gradients lives in the
 * workspace, so concurrent backward calls need distinct workspaces.          */
int gs_render_backward(const gs_scene *scene, const gs_camera *camera, const float *bg,
                       void *workspace, size_t ws_bytes, const float *dL_dimage,
                       const float *dL_dalpha, uint32_t grad_layer_mask, const gs_grads *grads,
                       float *contrib_sum, float *contrib_max, void *stream);

/* Contribution prune (Sec. 3.2.2): keep[i] = contrib_max[i] >= threshold;
 * *n_keep (device int64) = number kept; keep_index (device int32 [N], may be
 * NULL) receives the kept indices in ascending order in its first *n_keep
 * entries.  workspace: gs_prune_workspace_size(n) bytes (NULL allowed when
 * keep_index is NULL).                                                        */
int gs_prune_workspace_size(int64_t n, size_t *bytes);
int gs_contrib_prune(const float *contrib_max, int64_t n, float threshold, uint8_t *keep,
                     int32_t *keep_index, int64_t *n_keep, void *workspace, size_t ws_bytes,
                     void *stream);

/* ---- Training step (Sec. 3.2: each layer is optimised with the layers below
 * it frozen, a random background colour per frame and the alpha channel in
 * the loss).  These are the pieces around gs_render / gs_render_backward.  */

/* Image loss and its gradient, all device float32, row-major planes:
 *   Y = target_rgb + (1 - target_alpha) bg        target under this frame's bg
 *   loss = (1 - lambda_dssim) mean|image - Y|
 *        + lambda_dssim (1 - mean SSIM(image, Y))
 *        + w_alpha mean|alpha - target_alpha|
 * image, target_rgb [3][H][W] (target_rgb premultiplied, without background),
 * alpha, target_alpha [H][W]; alpha may be NULL (no alpha term; then
 * dL_dalpha, if given, is zeroed).  SSIM (Wang et al. 2004) per channel with
 * an 11x11 Gaussian window of sigma 1.5, zero outside the image, C1 = 1e-4,
 * C2 = 9e-4.  Writes *loss (device float), dL_dimage [3][H][W] and, when not
 * NULL, dL_dalpha [H][W].  workspace: gs_image_loss_workspace_size bytes
 * (9 W H floats of per-pixel maps plus block sums), 256-byte aligned.
 * Asynchronous; GS_ERR_INVALID for NULL inputs or bad sizes.                 */
int gs_image_loss_workspace_size(int32_t width, int32_t height, size_t *bytes);
int gs_image_loss(const float *image, const float *alpha, const float *target_rgb, const float *target_alpha,
                  const float *bg, int32_t width, int32_t height, float lambda_dssim, float w_alpha,
                  void *workspace, size_t ws_bytes, float *loss, float *dL_dimage, float *dL_dalpha,
                  void *stream);

/* Adam moments (device float32, shaped like the gs_grads fields), in the
 * order means, log_scales, quats, opacity_logit, sh.                        */
typedef struct gs_adam_state {
    float *m[5];
    float *v[5];
} gs_adam_state;

/* One Adam step (Kingma & Ba 2015, with bias correction) on the scene's
 * parameters IN PLACE (the scene's pointers are written despite the const
 * of gs_scene; every field must be float32).  lr[5] per field in the order
 * of gs_adam_state; step t >= 1 is this update's index.  A Gaussian whose
 * layer bit is not in train_layer_mask keeps parameters and moments
 * (frozen layers).  GS_ERR_INVALID for non-float32 fields or NULL arrays.   */
int gs_adam_step(const gs_scene *scene, const gs_grads *grads, const gs_adam_state *state, const float *lr,
                 float beta1, float beta2, float eps, int32_t step, uint32_t train_layer_mask, void *stream);

/* Activity of the inactive pruning (Sec. 3.2.2), called after gs_adam_step
 * with the same state and hyper-parameters: for every Gaussian whose layer is
 * in train_layer_mask,
 *   activity[g] += 2 |d mean| + 0.1 |d SH| + 0.1 |d log-scale|
 * where d is the update that Adam step applied (recomputed from the moments
 * in state: m[0], v[0] means, m[4], v[4] SH, m[1], v[1] log-scales).  layer
 * u8 [n], activity f32 [n] (device, accumulated).  lr[5] as for gs_adam_step.
 * Asynchronous; GS_ERR_INVALID for NULL arrays or bad sizes.               */
int gs_activity_accumulate(const gs_adam_state *state, const uint8_t *layer, int64_t n, int32_t sh_degree,
                           const float *lr, float beta1, float beta2, float eps, int32_t step,
                           uint32_t train_layer_mask, float *activity, void *stream);

/* Inactive pruning decision (Sec. 3.2.2): keep[i] = 0 when layer i is in
 * train_layer_mask and activity[i] / samples <= threshold (the average over
 * the samples accumulated since the last decision), else 1; keep_index and
 * n_keep as for gs_contrib_prune, with its workspace size.  The caller
 * multiplies the threshold by the decay (0.975 in the paper) after each
 * decision and resets activity.                                              */
int gs_activity_prune(const float *activity, const uint8_t *layer, int64_t n, uint32_t train_layer_mask,
                      float samples, float threshold, uint8_t *keep, int32_t *keep_index, int64_t *n_keep,
                      void *workspace, size_t ws_bytes, void *stream);

/* ---- SH codebook construction (Sec. 3.3, K-means; offline, before rendering)
 * Points are rows of `dim` <= 48 floats, `stride` floats apart (device).
 * gs_kmeans_assign: assign[i] = argmin_j |x_i - c_j|^2 over the k centroids
 * (float32 [k][dim], device), ties to the lower index.
 * gs_kmeans_update: every centroid with at least one assigned point becomes
 * their mean; scratch: gs_kmeans_scratch_size bytes (device).
 * gs_sh_codebook_encode: from a float32 scene's sh [N][K][3] and the final
 * assignment and centroids (dim = 3(K-1), the coefficients k >= 1): dc
 * float32 [N][3], index uint16 [N] (k <= 65536), table FP16 [k][R] as
 * described at gs_scene.  All asynchronous.                                 */
int gs_kmeans_scratch_size(int32_t k, int32_t dim, size_t *bytes);
int gs_kmeans_assign(const float *points, int64_t n, int32_t dim, int64_t stride, const float *centroids, int32_t k,
                     uint32_t *assign, void *stream);
int gs_kmeans_update(const float *points, int64_t n, int32_t dim, int64_t stride, const uint32_t *assign, int32_t k,
                     float *centroids, void *scratch, size_t scratch_bytes, void *stream);
int gs_sh_codebook_encode(const float *sh, int64_t n, int32_t sh_degree, const uint32_t *assign,
                          const float *centroids, int32_t k, float *dc, uint16_t *index, void *table, void *stream);

/* Row gather for applying a prune: dst row i = src row index[i] for
 * i < n, rows of row_bytes > 0 bytes (2-byte aligned arrays when row_bytes is
 * even; copied in 4-, 2- or 1-byte words); index (device int32) as written
 * by gs_contrib_prune's keep_index, every entry a valid row of src.  dst must
 * not overlap src.  Asynchronous.                                            */
int gs_gather_rows(const void *src, void *dst, int64_t row_bytes, const int32_t *index, int64_t n, void *stream);

/* Byte offsets of the regions of a render workspace of ws_bytes bytes, for
 * tests and debugging tools (host only, no device access).  out[k] for
 * k = 0..GS_LAYOUT_COUNT-1 in this order:
 *   0 status/control block   1 records (48 B per Gaussian: u, v, A2, beta,
 *   G2, opacity, r, g, b, depth, rect01, rect23)   2 tiles touched (u32)
 *   3 depth keys (u32 float bits, 0xFFFFFFFF when culled)   4 the pair list:
 *   Gaussian ids (u32) in tile order, depth order within a tile   5 tile
 *   ranges (u32 start, end per tile)   6 final transmittance (f32 per pixel)
 *   7 n_contrib (u32 per pixel)   8 record gradients (48 B per Gaussian)
 *   9 total bytes   10 pair capacity.  Returns GS_ERR_WORKSPACE when
 *   ws_bytes is below the fixed part.                                         */
#define GS_LAYOUT_COUNT 11
int gs_workspace_layout(int64_t n, int32_t width, int32_t height, size_t ws_bytes, int64_t *out);

/* gs_contrib_prune without a workspace, for callers that cannot allocate
 * device memory: code running inside a host application's frame callback or
 * plugin (a game engine or VR compositor render thread) where a device
 * allocation would stall every stream or is forbidden outright, and code that
 * must not touch the allocator at all between set-up and shutdown.  The paper
 * has no counterpart; this is an interface convenience of this library.
 * Same arguments and results as gs_contrib_prune minus the workspace.  The
 * scan scratch (8 KiB, of which the scan uses one 32-bit partial count per
 * scan block, at most 1024) is a static device array in the library, held
 * by every GPU that loads the library until the process exits; no
 * cudaMalloc/cudaFree or allocating library routine is called.  n must be
 * in 0 .. 2^31-1 (GS_ERR_INVALID otherwise).  Every call looks up the
 * array's device address (cudaGetSymbolAddress) with the calling thread's
 * current device, so the address stays right after a device reset.  The
 * first call on each device also loads the library's module on that device,
 * and that load is when the driver backs the array with device memory: a
 * caller that may not allocate later makes one warm-up call (n = 0 is
 * enough) on each device at set-up, before any stream capture.  Every call
 * shares the one array, so calls that overlap on the GPU (different streams,
 * or host threads without ordering) race.                                    */
int gs_contrib_prune_noalloc(const float *contrib_max, int64_t n, float threshold, uint8_t *keep,
                             int32_t *keep_index, int64_t *n_keep, void *stream);

/* Copies the status word of a render workspace to host memory and
 * synchronises the stream.                                                   */
int gs_read_status(const void *workspace, gs_status *out, void *stream);

/* Stage timing.  When enabled, every entry point records a CUDA event pair
 * around each of its stages on the call's stream (no synchronisation).
 * gs_profile_collect waits for the recorded events, adds each stage's elapsed
 * milliseconds and call count since the previous collect to ms[k] and
 * calls[k] (arrays of GS_STAGE_COUNT, host), and resets.  Disabled by default;
 * stage k's kernels per call are listed in kernels[k] when non-NULL.
 * Not thread safe: enable it in one thread at a time.                        */
enum {
    GS_STAGE_PREPROCESS = 0,   /* S1 */
    GS_STAGE_COMPACT,          /* S2: visible count, digit histograms and first-digit tile counts of the depth keys */
    GS_STAGE_DEPTH_SORT,       /* S2: radix digit kernels on the depth bits (the first compacts) */
    GS_STAGE_BIN_ROWS,         /* S2: depth-ordered split of the pairs into tile rows */
    GS_STAGE_BIN_TILES,        /* S2: split of every row into its tiles, tile ranges */
    GS_STAGE_COMPOSITE_SETUP,  /* S3/S4: compositor set-ups (forward tile order and checkpoint bases;
                                  backward: zeroed record gradients; the forward writes the backward's
                                  work items) */
    GS_STAGE_COMPOSITE,        /* S3 (one launch per gs_render or gs_render_batch call) */
    GS_STAGE_COMPOSITE_BWD,    /* S4a: the backward compositor */
    GS_STAGE_PREPROCESS_BWD,   /* S4b */
    GS_STAGE_PRUNE,            /* S5 */
    GS_STAGE_LOSS,             /* training: image loss and its gradient */
    GS_STAGE_ADAM,             /* training: parameter update */
    GS_STAGE_COUNT
};
int gs_profile_enable(int on);
int gs_profile_collect(double *ms, int64_t *calls);
/* Kernels launched by the library since it was loaded (all entry points). */
int64_t gs_kernel_launches(void);

/* The method's constants as this library applies them (Sec. 3.3 renders the
 * splats as the cited 3DGS renderer does; these are its values): tile edge,
 * EWA dilation of the 2D covariance (px^2), alpha clamp and skip threshold,
 * early-stop transmittance, frustum clamp factor, radius in standard
 * deviations and the eigenvalue floor, the backward checkpoint stride, and
 * the limits of one call.  Host only.                                        */
typedef struct gs_settings {
    int32_t tile;                 /* 16 */
    float dilation;               /* 0.3 */
    float alpha_max;              /* 0.99 */
    float alpha_min;              /* 1/255 */
    float t_min;                  /* 1e-4 */
    float frustum_clamp;          /* 1.3 */
    float radius_sigmas;          /* 3 */
    float eigen_floor;            /* 0.1 */
    int32_t checkpoint_stride;    /* list positions between backward checkpoints (256) */
    int32_t max_sh_degree;        /* 3 */
    int32_t max_planes;           /* GS_MAX_PLANES */
    int32_t max_image_dim;        /* GS_MAX_IMAGE_DIM */
    int32_t max_batch;            /* GS_MAX_BATCH */
    int32_t debug_build;          /* 1 when compiled with GS_DEBUG */
} gs_settings;
int gs_get_settings(gs_settings *out);

/* ---- GS_DEBUG builds (libgs_debug.so; the paper has no counterpart) ----
 * A library compiled with GS_DEBUG checks, inside its kernels, the indices it
 * writes and reads against the sizes they index: tile rectangles against the
 * tile grid, depth-sort scatter positions against the visible count, row-list
 * and pair-list positions against the pair capacity, tile ranges against the
 * pair count, Gaussian ids read from the lists against the Gaussian count,
 * checkpoint segments against the checkpoint area.  A failed check skips the
 * access, sets GS_ERR_BOUNDS in the workspace status word (first failure
 * wins) and records which check failed; it never traps.  In a release build
 * the checks compile to nothing.
 *   gs_debug_build():  1 in a GS_DEBUG build, 0 otherwise.
 *   gs_debug_site():   copies the number of the first failed check of the
 *                      workspace's last render to *site (host; 0 = none) and
 *                      synchronises the stream.  GS_ERR_INVALID in release.
 *   gs_debug_sort_wait(): test hook of the depth sort's bounded look-back
 *                      wait.  spin_limit replaces its iteration limit
 *                      (0 restores the default); withhold_pass >= 1 makes the
 *                      first tile of that digit kernel never publish its
 *                      counts, so the tiles after it wait until the limit
 *                      runs out and write GS_ERR_TIMEOUT to the status word
 *                      (-1 disables).  After a timeout the binning does not
 *                      read the unfinished order: the render draws nothing
 *                      and the status holds the error.  Process-wide, not
 *                      thread safe; GS_ERR_INVALID in release builds.        */
int gs_debug_build(void);
int gs_debug_site(const void *workspace, uint32_t *site, void *stream);
int gs_debug_sort_wait(uint32_t spin_limit, int32_t withhold_pass);

/* Message of the calling thread's last error ("" if none). */
const char *gs_last_error_string(void);

/* Library version string. */
const char *gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
