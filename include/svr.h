/*
 * svr.h - C ABI of the sparse-voxel rasterizer for one GB300 (sm_103a).
 *
 * Hot path of SVRaster (Sun et al., "Sparse Voxels Rasterization: Real-time
 * High-fidelity Radiance Field Rendering", arXiv 2412.04459):
 *
 *   svr_preprocess  per view: ray sign masks of the 16x16 tiles and, per
 *                   voxel, its Morton code, its tile rectangle, its colour
 *                   and its 8 corner densities (Sec. 3.1.2 "Projection to
 *                   image space", "Pre-processing voxels"; Sec. A.1, Sec. B.1)
 *   svr_bin_sort    one (key, value) pair per (voxel, tile, ray sign
 *                   pattern), sorted by (tile, direction-dependent Morton
 *                   order), and the range of each tile (Sec. 3.1.2 "Sorting
 *                   voxels"; Sec. B.1, Sec. B.2)
 *   svr_render_fwd  per pixel front-to-back compositing of its tile's list
 *                   (Eq. alpha_blend, Eq. vox_alpha, Eq. vox_color, Sec. A.2,
 *                   Sec. A.4; early termination, Sec. 3.1.2)
 *   svr_render_bwd  gradients of the three images with respect to the grid
 *                   point densities and the SH coefficients (Sec. A.2, A.4)
 *
 * Conventions shared by every call
 *   - Array arguments are DEVICE pointers owned by the caller, row-major and
 *     contiguous, valid until the last call that uses them has finished on
 *     the stream.  The library allocates no device or pinned memory: all
 *     scratch lives in the caller's workspace (svr_workspace_size bytes,
 *     256-byte aligned).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only
 *     enqueue work, except where a description says it synchronises.
 *   - Return value: SVR_OK or an SVR_ERR_* code; svr_last_error() gives a
 *     message for the calling thread.  Argument errors are found on the host
 *     before anything is enqueued.  Errors found by kernels (an invalid
 *     voxel, too many pairs) are recorded in the workspace and reported by
 *     svr_frame_status(), or by svr_bin_sort() when it is asked for the
 *     pair count.
 *   - Camera: OpenCV pinhole.  Camera point X = R p + t with w2c = [R | t]
 *     row-major; pixel (x, y) has its centre at (x + 0.5, y + 0.5); the ray
 *     of a pixel is r_o + t r_d with r_o = -R^T t and r_d = R^T ((x + .5 -
 *     cx) / fx, (y + .5 - cy) / fy, 1), so ray distances are camera depths.
 *   - Voxel (Eq. vox_coord): level l in [1, 16], size v_s = w_s 2^-l, centre
 *     on the lattice w_c - w_s/2 + v_s (ijk + 1/2) (read as the cell centre).
 *     Corner j of a voxel has offsets (j>>2 &1, j>>1 &1, j &1) in (x, y, z),
 *     the V_000 ... V_111 order of Eq. interp.  Grid point values are raw
 *     densities; explin is applied after trilinear interpolation.
 *   - SH: degree 3, sh[v][n][c] (16 coefficients x RGB, coefficient-major),
 *     real orthonormal basis without the Condon-Shortley phase, index n =
 *     l*l + l + m; colour = max(0, sum_n Y_n(d) sh[v][n][c]) with d =
 *     normalize(centre - r_o) (Eq. vox_color).
 */
#ifndef SVR_H_
#define SVR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SVR_API __attribute__((visibility("default")))
#else
#define SVR_API
#endif

#define SVR_OK 0
#define SVR_ERR_INVALID 1  /* bad argument, or a voxel off its lattice / level outside [1, max_level] */
#define SVR_ERR_LIMIT 2    /* more than 2^29 voxels or 2^16 tiles (the key layout of Sec. B.1) */
#define SVR_ERR_CAPACITY 3 /* more pairs than the workspace holds; the true count is reported */
#define SVR_ERR_CUDA 4     /* a CUDA runtime call failed */
#define SVR_ERR_TIMEOUT 5  /* a bounded device wait gave up */

/* Device-side error flags (svr_frame_status). */
#define SVR_FLAG_INVALID_VOXEL 1u
#define SVR_FLAG_CAPACITY 2u
#define SVR_FLAG_NO_FORWARD 4u /* svr_render_bwd ran before any svr_render_fwd of the sort (or, with
                                  d_normal or d_distortion, before one that rendered normals or the
                                  distortion loss: then the split tiles are skipped) */

typedef struct svr_camera {
    float fx, fy, cx, cy;
    float w2c[12]; /* row-major [R | t] */
    int32_t width, height;
} svr_camera;

typedef struct svr_params {
    int32_t K;      /* samples per ray segment, 1..3 (Eq. K_samp_pts) */
    float t_stop;   /* stop compositing once T < t_stop (Sec. 3.1.2; 1e-4 in the paper) */
    int32_t tile;   /* tile edge in pixels: 16 as in the paper (Sec. B.1), or 8 or 32 */
    float bg[3];    /* background colour added as T_final * bg */
} svr_params;

/* Views rendered together by svr_preprocess_views / svr_render_batched. */
#define SVR_MAX_VIEWS 32

typedef struct svr_scene {
    float world_center[3]; /* w_c */
    float world_size;      /* w_s */
    int64_t n_vox;         /* N, at most 2^29 */
    int64_t n_pts;         /* number of grid points */
    int32_t max_level;     /* upper bound on level[], 1..16; sets the sorted key width */
    int32_t reserved;
    const float *centre;       /* [N][3] */
    const uint8_t *level;      /* [N] */
    const int32_t *corner_idx; /* [N][8], indices into grid */
    const float *grid;         /* [n_pts] raw densities */
    const float *sh;           /* [N][48], 16-byte aligned */
} svr_scene;

/*
 * State of one view or a batch of views, in HOST memory owned by the caller.
 * svr_preprocess / svr_preprocess_views fill it; svr_bin_sort,
 * svr_render_fwd and svr_render_bwd read it (svr_bin_sort also updates it).
 * It points into the workspace and at the scene arrays, which must stay
 * alive while it is used.  Treat the fields as read-only.
 *
 * Tiles of all views share one numbering: view v owns global tiles
 * [tile_base[v], tile_base[v+1]), its tile (tx, ty) being tile_base[v] +
 * ty * ntx_v + tx.  Images of all views share one buffer per output: view v
 * owns pixels [pixel_base[v], pixel_base[v+1]) of depth/alpha/T_final/last
 * (row-major H_v x W_v) and floats [3 pixel_base[v], 3 pixel_base[v+1]) of
 * rgb (planar [3][H_v][W_v]).
 */
typedef struct svr_frame {
    svr_scene scene;
    svr_params params;
    int32_t n_views;     /* 1 after svr_preprocess */
    int32_t key_shift;   /* Morton bits under the tile id in a key: 48 for svr_preprocess */
    int64_t total_tiles;
    svr_camera cams[SVR_MAX_VIEWS];
    int32_t tile_base[SVR_MAX_VIEWS + 1];
    int64_t pixel_base[SVR_MAX_VIEWS + 1];
    double ray_origin[SVR_MAX_VIEWS][3];
    void *ws;
    size_t ws_bytes;
    int64_t pair_capacity;
    int64_t n_pairs;    /* pair count, or -1 while it is known only on the device */
    int32_t stage;      /* 1 after preprocessing, 2 after svr_bin_sort */
    int32_t sorted_alt; /* internal: which key buffer holds the sorted pairs */
    uint64_t offsets[24]; /* internal: byte offsets of the workspace buffers */
} svr_frame;

/* Device views of the internal buffers of a frame, for inspection. */
typedef struct svr_buffers {
    const void *status;       /* uint32[16]: flags, n_pairs (low, high), ... */
    const uint8_t *tile_mask; /* [total_tiles] bit s set if a pixel of the tile has ray sign bits s */
    const uint64_t *octpath;  /* [N] Morton code (Sec. A.1) */
    const int16_t *rect;      /* [V][N][4] tx0, tx1, ty0, ty1 (empty: tx0 > tx1) */
    const uint32_t *count;    /* [V][N] pairs emitted per (view, voxel) */
    const uint32_t *offset;   /* NULL: pairs are written per tile, not at per-voxel offsets */
    const float *record;      /* [V][N][16] per-voxel record of each view */
    const uint64_t *keys;     /* [pair_capacity] sorted keys: tile << key_shift | Morton order */
    const uint32_t *values;   /* [pair_capacity] sorted values: s << 29 | voxel id */
    const uint32_t *ranges;   /* [total_tiles][2] begin, end of each tile's list */
} svr_buffers;

/* Workspace bytes needed for n_vox voxels, pair_capacity pairs and this
 * camera / tile size; 0 if the arguments are invalid.  Host only. */
SVR_API size_t svr_workspace_size(int64_t n_vox, int64_t pair_capacity,
                                  const svr_camera *cam, const svr_params *params);

/* Workspace bytes for a batch of n_views (1..SVR_MAX_VIEWS) cameras. */
SVR_API size_t svr_workspace_size_views(int64_t n_vox, int64_t pair_capacity,
                                        const svr_camera *cams, int n_views,
                                        const svr_params *params);

/*
 * Per-view preprocessing (Sec. 3.1.2 "Projection to image space" and
 * "Pre-processing voxels").  Enqueues:
 *   - per tile, the 8-bit mask of ray sign patterns 4(rd.x<0) + 2(rd.y<0) +
 *     (rd.z<0) of its in-image pixels (Sec. B.2 listing, Sec. B.1);
 *   - per voxel: lattice index and Morton code (Sec. A.1); the tile
 *     rectangle of the 2-D bounding box of its 8 projected corners (all
 *     corners at camera depth <= 1e-3: culled; some: whole image); the pair
 *     count = sum over the rectangle's tiles of the number of sign patterns
 *     in the tile mask; its colour (Eq. vox_color) and its 8 gathered corner
 *     densities.
 * Fills *frame.  pair_capacity: pairs the workspace was sized for.
 * Errors: SVR_ERR_INVALID (null pointer, K not in 1..3, tile != 16, bad
 * camera, misaligned sh or workspace, workspace too small, max_level outside
 * 1..16), SVR_ERR_LIMIT (N > 2^29, more than 2^16 tiles), SVR_ERR_CUDA.
 */
SVR_API int svr_preprocess(svr_frame *frame, const svr_scene *scene, const svr_camera *cam,
                           const svr_params *params, void *ws, size_t ws_bytes,
                           int64_t pair_capacity, void *stream);

/*
 * svr_preprocess for a batch of n_views (1..SVR_MAX_VIEWS) views of one scene
 * rendered together: the views' tiles are numbered consecutively (see
 * svr_frame), all pairs of all views are sorted at once and one persistent
 * launch composites every (view, tile) of the batch.  Per view the result is
 * that of svr_preprocess; the sorted order within each (view, tile) is the
 * paper's.  The keys are compact: tile id << S | the top S bits of the
 * direction-dependent Morton order, S = 3 min(16, max_level + 1), so the
 * tile ids of all views need only fit 64 - S bits (SVR_ERR_LIMIT otherwise).
 * The paper renders one view at a time; batching is this library's addition.
 */
SVR_API int svr_preprocess_views(svr_frame *frame, const svr_scene *scene, const svr_camera *cams,
                                 int n_views, const svr_params *params, void *ws, size_t ws_bytes,
                                 int64_t pair_capacity, void *stream);

/*
 * Pair emission and sort (Sec. B.1).  Enqueues: the exclusive scan of the
 * per-tile pair counts (counted by svr_preprocess), which gives every tile
 * its [begin, end) range of the pair list; one pair per (voxel, tile of its
 * rectangle, sign pattern s of that tile) written into that tile's range,
 * key = tile << 48 | (octpath XOR s replicated in all 16 triples) (the
 * direction-dependent Morton order of Sec. B.2), value = s << 29 | voxel id;
 * then a sort of each tile's range by the Morton bits that can differ (the
 * top 3 (max_level + 1) of the 48; with max_level = 16 all of them and the
 * value first), done tile by tile in shared memory: stable LSD radix sorts of
 * 1024-pair chunks, whose runs are merged per tile.  The result equals a sort
 * of all pairs by (key, value): within a tile distinct pairs have distinct
 * (key, value).  Also builds the render work order and the per-block lists.
 * n_pairs_out: if not NULL, the call synchronises the stream, stores the
 * true pair count there, and returns SVR_ERR_CAPACITY if it exceeds the
 * capacity (no pair was written; re-run with a larger workspace) or
 * SVR_ERR_INVALID if a voxel failed its lattice or level check.  If NULL the
 * call only enqueues work (CUDA-graph capturable) and such errors are left
 * for svr_frame_status().
 */
SVR_API int svr_bin_sort(svr_frame *frame, int64_t *n_pairs_out, void *stream);

/*
 * Forward render (Sec. 3.1.2 "Rendering pixels").  Per pixel, its tile's
 * sorted list is walked front to back; entries with other sign bits are
 * skipped (Sec. B.1); for a valid ray-AABB segment [a, b] (Sec. A.2) the
 * voxel alpha uses K samples t_k = a + (k - 1/2)(b - a)/K, trilinear raw
 * density, explin, alpha = 1 - exp(-(l/K) sum_k explin(v_k)), l = (b - a)|r_d|
 * (Eq. supp_alpha_comp); the voxel depth is sum_k prod_{j<k}(1 - a_j) a_k t_k
 * (Sec. A.4); C += T alpha c, D += T d, T *= 1 - alpha; the walk stops after
 * the voxel that leaves T < t_stop.
 * Outputs (device, caller-owned): rgb [3][H][W] = C + T_final bg, depth
 * [H][W], alpha [H][W] = 1 - T_final, T_final [H][W], last [H][W] = index in
 * the sorted pair list of the voxel that stopped the walk, else the tile's
 * last entry (-1 for an empty tile).  T_final and last are what
 * svr_render_bwd needs.  Requires svr_bin_sort first.
 */
SVR_API int svr_render_fwd(const svr_frame *frame, float *rgb, float *depth, float *alpha,
                           float *T_final, int32_t *last, void *stream);

/*
 * Backward render (Sec. A.2 alpha gradient, Sec. A.4 depth gradients).
 * Inputs: dL/drgb [3][H][W], dL/ddepth [H][W], dL/dalpha [H][W] (any may be
 * NULL = zero) and the T_final, last of svr_render_fwd.  Each pixel walks its
 * list back to front from `last`, recovering T before each voxel as T after
 * it divided by (1 - alpha); pixels with T_final < 1e-30 redo the walk front
 * to back instead.  Adds dL/dgrid into d_grid [n_pts] (accumulated: the
 * caller zeroes it) and writes dL/dsh into d_sh [N][48] (zero for voxels not
 * in view).  Requires svr_render_fwd's outputs for the same frame, and that
 * the frame's last svr_render_fwd (or svr_render_stats) ran after its last
 * svr_bin_sort on the same stream: the forward leaves in the workspace each
 * pixel's hit masks over the batches of list entries it walked (the backward
 * takes its hits from them instead of testing the rays again) and, for tile
 * lists longer than 1024 entries, which are composited in segments, each
 * segment's transmittance and the colour and depth sums behind it, where the
 * backward starts from them.  Without such a forward every tile is skipped
 * and SVR_FLAG_NO_FORWARD is raised.
 */
SVR_API int svr_render_bwd(const svr_frame *frame, const float *d_rgb, const float *d_depth,
                           const float *d_alpha, const float *T_final, const int32_t *last,
                           float *d_grid, float *d_sh, void *stream);

/*
 * Whole batched step in one call: svr_preprocess_views, svr_bin_sort without
 * a pair count (no host synchronisation), svr_render_fwd and, when d_rgb,
 * d_depth or d_alpha is not NULL, svr_render_bwd.  Only enqueues work, so the
 * call can be captured in a CUDA graph and replayed (inputs and outputs must
 * then stay at the same addresses).  Outputs and gradients use the batch
 * layout of svr_frame; d_grid accumulates over all views, d_sh sums the views.
 * Capacity overflow or invalid voxels are reported by svr_frame_status.  The
 * paper has no batched path; see svr_preprocess_views.
 */
SVR_API int svr_render_batched(svr_frame *frame, const svr_scene *scene, const svr_camera *cams,
                               int n_views, const svr_params *params, void *ws, size_t ws_bytes,
                               int64_t pair_capacity, float *rgb, float *depth, float *alpha,
                               float *T_final, int32_t *last, const float *d_rgb,
                               const float *d_depth, const float *d_alpha, float *d_grid,
                               float *d_sh, void *stream);

/*
 * Extra outputs and inputs of svr_render_fwd_ex / svr_render_bwd_ex.  Any
 * member may be NULL (not computed / zero).  Device pointers, caller-owned,
 * 4-byte aligned.
 *   normal      forward output, planar [3][H][W] like rgb (batch layout for
 *               a batch): N = sum_i T_i alpha_i n_i, the voxel normal n =
 *               normalize(gradient of the trilinear density field at the
 *               voxel centre) in world axes (Eq. vox_normal, closed form of
 *               Eq. interp_grad; the zero vector where the gradient
 *               vanishes), composited like colour with no background term.
 *   max_weight  forward output [N]: raised (atomic max, never lowered) to
 *               every voxel's largest blending weight T_i alpha_i over the
 *               rendered pixels: the pruning statistic of Sec. 3.2.2,
 *               accumulated over views and calls until the caller zeroes it.
 *               The later segments of tile lists longer than 1024 entries
 *               are walked a second time, in parallel, from the true
 *               transmittance in front of them, to get it exactly.  Given to
 *               svr_render_bwd_ex, the backward raises it too, from the
 *               exact T_i alpha_i of its own walk at no extra pass (a
 *               training loop gets the pruning statistic with its gradients).
 *   d_normal    backward input [3][H][W]: dL/dN.  Requires that the frame's
 *               last forward of this sort rendered `normal` (its tile
 *               segments carry the normal sums); otherwise split tiles are
 *               skipped and SVR_FLAG_NO_FORWARD is raised.  The gradient
 *               passes the normalisation and Eq. interp_grad_grad into d_grid.
 *   priority    backward output [N]: accumulates (adds to) every voxel's
 *               subdivision priority sum over pixels |alpha_i dL/dalpha_i|
 *               (Eq. priority), dL/dalpha_i the derivative of the objective
 *               (the upstream gradients of all images, normals included) with
 *               respect to the voxel's alpha in the compositing of Eq.
 *               alpha_blend, its colour, normal and depth held fixed.
 *   distortion  forward output [2][H][W] (batch: 2 planes per view, at
 *               2 pixel_base[v]): plane 0 the distortion loss of each ray
 *               (Sec. 3.2.3, the loss of Mip-NeRF 360) over its composited
 *               voxels, L = sum_ij w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2
 *               delta_i with w_i = T_i alpha_i, m_i = (a_i + b_i) / 2 and
 *               delta_i = b_i - a_i in ray distance (camera depth); plane 1
 *               sum_i w_i m_i, which the backward needs.  Also read by the
 *               backward when d_distortion is set.
 *   d_distortion backward input [H][W]: dL/dL_dist per ray (e.g. the loss
 *               weight over the pixel count).  Requires `distortion` from
 *               the frame's last forward of this sort (split tiles carry the
 *               distortion sums; otherwise they are skipped and
 *               SVR_FLAG_NO_FORWARD is raised).
 */
typedef struct svr_render_extras {
    float *normal;
    float *max_weight;
    const float *d_normal;
    float *priority;
    float *distortion;
    const float *d_distortion;
} svr_render_extras;

/* svr_render_fwd plus the forward members of *extras (NULL: none). */
SVR_API int svr_render_fwd_ex(const svr_frame *frame, float *rgb, float *depth, float *alpha,
                              float *T_final, int32_t *last, const svr_render_extras *extras,
                              void *stream);

/* svr_render_bwd plus the backward members of *extras (NULL: none). */
SVR_API int svr_render_bwd_ex(const svr_frame *frame, const float *d_rgb, const float *d_depth,
                              const float *d_alpha, const float *T_final, const int32_t *last,
                              float *d_grid, float *d_sh, const svr_render_extras *extras,
                              void *stream);

/* svr_render_fwd that also writes, per pixel, counts[y][x] = (list entries
 * with the pixel's sign bits that it examined, hits it composited): the
 * work the forward did, for throughput accounting.  counts: device int32
 * [H][W][2], 8-byte aligned.  Slower than svr_render_fwd; same images. */
SVR_API int svr_render_stats(const svr_frame *frame, float *rgb, float *depth, float *alpha,
                             float *T_final, int32_t *last, int32_t *counts, void *stream);

/*
 * Forward render of one view that allocates nothing and needs no workspace
 * from the caller.  The paper has no counterpart: it exists for callers that
 * may not allocate device memory themselves (a plugin inside an application
 * that owns the device-memory budget, or a latency-critical render callback
 * where an allocation and the device synchronisation it can cause are not
 * allowed).  Same computation and outputs as svr_preprocess + svr_bin_sort
 * (with a pair count) + svr_render_fwd, but the scratch memory is one 16 MiB
 * array compiled into the library, which every GPU that loads the library
 * keeps until the process exits.
 * Limits: at most 65536 voxels, at most 2^16 tiles, and as many pairs as fit
 * in the array next to the voxel buffers; beyond them the call returns
 * SVR_ERR_LIMIT (voxels, tiles or image) or SVR_ERR_CAPACITY (pairs; the
 * render is skipped and *n_pairs_out holds the true count).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the
 * process: do not use the library across a cudaDeviceReset.  Every call
 * synchronises the stream (it reads the pair count back, like svr_bin_sort
 * with a count), so it cannot be called while the stream is being captured
 * into a CUDA graph.  All calls share the array and each leaves its contents
 * behind (everything that must start at zero is cleared by the call); calls
 * whose GPU work overlaps race on the array.  Outputs as for svr_render_fwd;
 * n_pairs_out may be NULL.
 */
SVR_API int svr_render_fwd_static(const svr_scene *scene, const svr_camera *cam,
                                  const svr_params *params, float *rgb, float *depth,
                                  float *alpha, float *T_final, int32_t *last,
                                  int64_t *n_pairs_out, void *stream);

/*
 * Supersampling anti-aliasing (Sec. 3.1.2 "Anti-aliasing": render at h_ss
 * times the resolution, then downsample with an anti-aliasing filter).  The
 * caller renders the view with a camera of width_ss x height_ss pixels over
 * the same image plane (intrinsics scaled by width_ss / width and height_ss /
 * height; the paper uses h_ss = 1.1 .. 1.5) and downsamples every output
 * plane with svr_downsample: target pixel (x, y) is the average of the
 * supersampled image over its footprint [s_x x, s_x (x + 1)) x [s_y y,
 * s_y (y + 1)), s_x = width_ss / width (area filter; the paper names no
 * filter).  src: device float [planes][height_ss][width_ss] (rgb: 3 planes,
 * depth, alpha: 1); dst: [planes][height][width].  Ratios must lie in [1, 4]
 * per axis (SVR_ERR_INVALID otherwise).  Enqueues only.
 */
SVR_API int svr_downsample(const float *src, int64_t planes, int height_ss, int width_ss, float *dst,
                           int height, int width, void *stream);

/* Backward of svr_downsample (its transpose): d_src [planes][height_ss][width_ss]
 * is overwritten with the gradient for the upstream d_dst [planes][height][width]. */
SVR_API int svr_downsample_bwd(const float *d_dst, int64_t planes, int height, int width, float *d_src,
                               int height_ss, int width_ss, void *stream);

/*
 * Mean squared error of a rendered image against a target, the MSE term of
 * the photometric loss (Sec. 3.2.3): *loss = sum_i (pred_i - target_i)^2 / n
 * and, if grad is not NULL, grad_i = 2 (pred_i - target_i) / n (the upstream
 * gradient for svr_render_bwd).  Device pointers: pred, target, grad [n],
 * loss one float (overwritten).  Enqueues only.
 */
SVR_API int svr_l2_loss(const float *pred, const float *target, int64_t n, float *grad,
                        float *loss, void *stream);

/*
 * Training-step pieces (Sec. 3.2.3 objectives; optimizer settings of the
 * supplementary's implementation details).  Device pointers; enqueue only.
 *
 * svr_t_concentration_loss: the transmittance-concentration loss L_T, which
 * pushes each ray's final transmittance T = 1 - alpha toward 0 or 1 (the
 * paper gives no formula; read as the binary entropy -(T ln T + (1 - T)
 * ln(1 - T)) with T clamped to [1e-6, 1 - 1e-6]).  Adds weight * mean over
 * the n pixels to *loss (the caller clears it, or svr_l2_loss wrote it) and,
 * if grad_alpha is not NULL, overwrites grad_alpha[i] with the gradient with
 * respect to alpha[i] (zero where the clamp acts).
 */
SVR_API int svr_t_concentration_loss(const float *alpha, int64_t n, float weight, float *grad_alpha,
                                     float *loss, void *stream);

/* Adds weight * mean(x[0..n)) to *loss (e.g. the distortion losses of the
 * rays from the distortion output of svr_render_fwd_ex, times lambda_dist). */
SVR_API int svr_weighted_mean(const float *x, int64_t n, float weight, float *loss, void *stream);

/*
 * One Adam step (Kingma and Ba) on n parameters: m = beta1 m + (1 - beta1) g,
 * v = beta2 v + (1 - beta2) g^2, param -= lr (m / (1 - beta1^step)) /
 * (sqrt(v / (1 - beta2^step)) + eps), with lr = lr_head for the elements whose
 * index modulo `period` is below `head` and lr_rest for the others (the SH
 * array [N][48]: period 48, head 3 gives the degree-0 coefficients their own
 * rate; the paper: 0.01 for them, 0.00025 for the rest, 0.025 for the grid
 * densities, (beta1, beta2) = (0.1, 0.99), eps = 1e-15).  step counts from 1;
 * m and v start at zero and are updated in place.  The four arrays must be
 * 16-byte aligned.  SVR_ERR_INVALID for a bad period/head/step, betas outside
 * [0, 1) or misaligned arrays.
 */
SVR_API int svr_adam(float *param, const float *grad, float *m, float *v, int64_t n, int32_t period,
                     int32_t head, float lr_head, float lr_rest, float beta1, float beta2, float eps,
                     int64_t step, void *stream);

/* Synchronises the stream and reads the device-side error flags
 * (SVR_FLAG_*) and the pair count of a frame.  Either output may be NULL. */
SVR_API int svr_frame_status(const svr_frame *frame, uint32_t *flags, int64_t *n_pairs,
                             void *stream);

/* Device pointers of a frame's internal buffers (valid while the frame is). */
SVR_API int svr_frame_buffers(const svr_frame *frame, svr_buffers *out);

/* Message of the last error on the calling thread ("" if none). */
SVR_API const char *svr_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
SVR_API int svr_version(void);

/* 1 if this library was built with SVR_DEBUG (libsvr_debug.so), else 0.
 * That build checks the data-dependent indices of the kernels' loads and
 * stores (tile ids < the frame's tiles, tile ranges within the pair capacity,
 * voxel ids of list entries < n_vox, corner indices of the gradient atomics
 * < n_pts, gradient-record and segment slots within their buffers, block
 * lists within their tile list or segment); a failed check skips the access
 * (a read takes index 0), is counted, and the first failure's site, index
 * and bound are kept.  Nothing traps.  (Corner indices of the scene are
 * validated in every build: svr_preprocess raises SVR_FLAG_INVALID_VOXEL.) */
SVR_API int svr_debug_build(void);

/* Waits for the current device, then writes its index-check report to
 * out[4] = {failed checks, site of the first (1 tile id, 2 tile range,
 * 3 voxel id, 4 gradient corner index, 5 record slot, 6 segment slot,
 * 7 block list length), its index, its bound} and clears it.
 * All zeros in builds without SVR_DEBUG.  out is a host array owned by the
 * caller; SVR_ERR_INVALID if it is NULL, SVR_ERR_CUDA on a CUDA error. */
SVR_API int svr_debug_report(uint64_t *out);

#ifdef __cplusplus
}
#endif

#endif /* SVR_H_ */
