/*
 * directl.h -- C ABI of the GB300 DirectL light-field renderer.
 *
 * DirectL (arXiv 2407.14053) renders a radiance field straight into the
 * encoded image of a lenticular light-field display: for every screen
 * subpixel it evaluates the interweave map (Sec. 3.1, Eqs. (1)-(3)), picks
 * the subpixel's ray after subpixel repurposing (Sec. 5, Alg. 2), and
 * composites 3D Gaussians front to back only for the rays and channels the
 * panel shows (Sec. 3.3, Eqs. (5), (8)-(10)).  Beside it the library builds
 * the paper's standard paradigm: render every view with a tile rasteriser,
 * then interweave (Alg. 1).
 *
 * Conventions for every call:
 *  - Return value: DL_OK (0) or a negative dl_status.  No call aborts the
 *    process or lets a C++ exception escape.  dl_last_error_detail() gives a
 *    one-line description of the last failure on a context.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Calls enqueue their device work on that stream.
 *    Calls that return sizes computed on the device (dl_set_display,
 *    dl_render_frame) synchronise `stream` once; see each call.
 *  - Ownership: the library owns scenes, display tables and its scratch
 *    memory (resident on the device until freed or the context is
 *    destroyed).  The caller owns every buffer it passes in; input buffers
 *    are only read during the call (they are copied), output buffers are
 *    written on `stream`.
 *  - Memory kinds: a pointer argument is device memory when the matching
 *    `*_on_device` flag is 1 and host memory when it is 0.
 *  - A context is bound to one device and is not thread-safe: callers that
 *    share a context between threads must serialise their calls.
 */
#ifndef DIRECTL_H
#define DIRECTL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dl_status;
enum {
    DL_OK = 0,
    DL_ERR_INVALID_ARG = -1,  /* a parameter is out of range or NULL        */
    DL_ERR_OOM = -2,          /* device or host allocation failed           */
    DL_ERR_CUDA = -3,         /* a CUDA runtime call failed                 */
    DL_ERR_NOT_FOUND = -4,    /* unknown scene or display id                */
    DL_ERR_TIMEOUT = -5,      /* a bounded device wait gave up              */
    DL_ERR_DEVICE_CHECK = -6, /* a kernel's own bounds check tripped        */
    DL_ERR_CAPACITY = -7      /* a frame needs more than 2^31-1 tile keys   */
};

/* Storage types of Gaussian attributes other than the means. */
enum { DL_F32 = 0, DL_BF16 = 1, DL_F16 = 2 };

/* Rendering paths. */
enum {
    DL_DIRECTL = 0,       /* repurposed rays only (Sec. 5 and Sec. 4)     */
    DL_STANDARD = 1,      /* all N_v views at panel resolution + Alg. 1   */
    DL_REQUIRED_ONLY = 2, /* identity ray assignment: blend only the pixels
                             the panel shows (Table 3, "Required Only")   */
    DL_RAYCAST = 3,       /* the rays of DL_DIRECTL cast through the scene:
                             ray-order 3DGS (Sec. 7, Alg. 3)              */
    DL_STANDARD_SR = 4    /* the paper's "HR w SR" baseline: all N_v views
                             at panel resolution as DL_STANDARD, then each
                             subpixel takes channel k of its view at its
                             repurposed source pixel (Sec. 5) instead of its
                             own pixel; equals DL_DIRECTL's image, computed
                             the standard way.  Tiles: DL_STANDARD's; the
                             DL_OPT_STANDARD_VIEW_SIZE option does not apply */
};

typedef struct dl_ctx dl_ctx;

/* Create a context on CUDA device `device`.  *out receives the handle. */
dl_status dl_create(dl_ctx** out, int32_t device);
/* Free every scene, display and scratch buffer of the context. */
dl_status dl_destroy(dl_ctx* ctx);
/* Static string naming a status code. */
const char* dl_status_string(dl_status s);
/* Copy the last error description (NUL-terminated, truncated to len). */
dl_status dl_last_error_detail(dl_ctx* ctx, char* buf, size_t len);

/*
 * 3D Gaussian scene, structure of arrays (Sec. 3.3: mean mu, covariance
 * Sigma = R S S^T R^T from a quaternion and per-axis log-scales, opacity,
 * spherical-harmonic colour).  Layouts: mean n*3 (always float32),
 * log_scale n*3, rot_wxyz n*4 (any length; normalised on use),
 * opacity_logit n (opacity = sigmoid(logit)), sh n*(d+1)^2*3 with the
 * coefficient index outer and RGB inner.  All but the means are stored in
 * `dtype` (DL_F32, DL_BF16 or DL_F16) as given.  1 <= n <= 2^28,
 * 0 <= sh_degree <= 3.
 */
typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t dtype;
    const float* mean;
    const void* log_scale;
    const void* rot_wxyz;
    const void* opacity_logit;
    const void* sh;
    int32_t on_device; /* 1: the five pointers are device memory */
} dl_gaussians_desc;

/* Copy a scene into library-owned device memory; *scene_id names it.
 * Enqueued on `stream`; the input may be reused once the call returns when
 * it is host memory, and once `stream` reaches this point when it is device
 * memory. */
dl_status dl_load_gaussians(dl_ctx* ctx, const dl_gaussians_desc* desc, void* stream,
                            int32_t* scene_id);
dl_status dl_free_scene(dl_ctx* ctx, int32_t scene_id);

/*
 * Lenticular display (Sec. 3.1 and Table 1).  width x height pixels of
 * three subpixels each; num_views = N_v; pitch_lx = line count L_x in
 * subpixel widths (0 < L_x <= 1024); tan_slant = tan(alpha) of the lens
 * tilt (|tan| <= 8); offset_k = K_offset in subpixel widths.  The map uses
 * these three rounded once to Q32 fixed point (round(3 tan 2^32),
 * round(L_x 2^32), round(K 2^32), nearest-even, in double precision); that
 * rounding is part of the display's definition and makes the map exact.
 * p_w = grating units per repurposing area (Sec. 5).  view_span_deg =
 * theta_d, the angle between the outermost cameras of the arc;
 * fov_x_deg = horizontal field of view of every camera.  repurpose = 1
 * applies Alg. 2, 0 gives every subpixel its own pixel.  reverse_views = 1
 * makes view 0 the rightmost camera.  rig selects the camera arrangement of
 * Sec. 3.2: 0 = cameras on an arc about the world origin, each looking at
 * it (T_v = R_y(-theta_v) L0); 1 = "off-axis perspective with straight
 * lines": L0 translated by x_v = D tan(theta_v) along its own x axis (D = the
 * depth of the world origin in L0's camera, which must be positive), all
 * axes parallel, each view's principal point shifted by f x_v / D columns
 * so that the plane at depth D has no parallax.  1 <= width, height <= 16384,
 * 1 <= num_views <= 65535.
 */
typedef struct {
    int32_t width, height, num_views, p_w;
    double pitch_lx, tan_slant, offset_k;
    double view_span_deg, fov_x_deg;
    int32_t repurpose, reverse_views;
    int32_t rig;
} dl_display_params;

/*
 * Build a display's offline tables on the device (the paper's offline step,
 * Sec. 4 step (1)): the view-index map V (Eqs. (1)-(3)), the repurposed
 * source pixel of every subpixel (Alg. 2) and the ray table (unique rays in
 * R-first order, Sec. 5).  Synchronises `stream` once to learn the ray
 * count.  *display_id names the result.
 */
dl_status dl_set_display(dl_ctx* ctx, const dl_display_params* params, void* stream,
                         int32_t* display_id);
dl_status dl_free_display(dl_ctx* ctx, int32_t display_id);
/* Number of rays N_rays and beta = N_rays / (w h) (either may be NULL). */
dl_status dl_display_info(dl_ctx* ctx, int32_t display_id, int64_t* n_rays, double* beta);

/* V, uint16, h rows of 3w entries: V[x*3w + 3y + k] = view of subpixel
 * (row x, column y, channel k) (Alg. 1, "Align with LCD panel"). */
dl_status dl_get_view_map(dl_ctx* ctx, int32_t display_id, uint16_t* out, int32_t out_on_device,
                          void* stream);
/* Encoded-image index matrix M_i (Sec. 5) as packed source pixels:
 * out[(x*w + y)*3 + k] = (x' << 16) | y' of the pixel of view V(x,3y+k)
 * whose channel k the subpixel shows. */
dl_status dl_get_subpixel_map(dl_ctx* ctx, int32_t display_id, uint32_t* out,
                              int32_t out_on_device, void* stream);
/* Ray table: ray_of[(x*w + y)*3 + k] = ray id of the subpixel (3wh
 * entries); rays[3*r .. 3*r+2] = (view, row, col) of ray r (N_rays*3
 * entries).  Rays are numbered in order of first use by the R subpixels
 * (row-major), then the G, then the B subpixels, so rays 0..wh-1 are the R
 * subpixels' rays whenever the three channels of every pixel show different
 * views.  Either output may be NULL. */
dl_status dl_get_ray_table(dl_ctx* ctx, int32_t display_id, uint32_t* ray_of, int32_t* rays,
                           int32_t out_on_device, void* stream);

/*
 * Render one encoded light-field frame (h x w x 3 float32, row-major,
 * RGB inner) of scene `scene_id` on display `display_id`.
 * L0_c2w: camera-to-world pose of the light-field centre, 4x4 row-major,
 * camera axes x right, y down, z forward (host memory, read during the
 * call).  View v's camera is T_v = R_y(-theta_v) L0 with theta_v =
 * -theta_d/2 + v theta_d/(N_v-1) (Eq. (17)).
 * mode: DL_DIRECTL, DL_STANDARD, DL_REQUIRED_ONLY, DL_RAYCAST or
 * DL_STANDARD_SR (see the mode enum).
 * out: h*w*3 floats, device memory if out_on_device else host memory (the
 * call then copies the frame back and returns once it is there).
 * Host synchronisation: the first DL_DIRECTL / DL_REQUIRED_ONLY frame of a
 * (scene, display, mode, tile shape) reads its key totals back to size the
 * tile-key buffer and the long-list capacity (one synchronisation of
 * `stream` in mid-frame); later frames of it are enqueued without any host
 * synchronisation, their launches sized from device counters.  Such a frame
 * that needs more tile keys or a longer list than those capacities is
 * dropped on the device: its output is left untouched and its status word
 * (dl_frame_stats.status, read by dl_last_frame_stats) is set; with a host
 * `out` the call sees this and renders the frame again, sized.  The next
 * frame after a dropped one, or after one that used more than 85 % of a
 * capacity, is sized again.  DL_STANDARD, DL_STANDARD_SR and frames on the
 * radix-sort fallback synchronise once per frame.
 */
dl_status dl_render_frame(dl_ctx* ctx, int32_t scene_id, int32_t display_id,
                          const double L0_c2w[16], int32_t mode, float* out,
                          int32_t out_on_device, void* stream);

/*
 * The frame of dl_render_frame, delivered to host memory without waiting for
 * it (Sec. 4 steps (2)-(3), as dl_render_frame): the frame's kernels run on
 * `stream`; its copy to `out` (host, h*w*3 floats; pinned, or the copy is
 * not asynchronous) is enqueued on `copy_stream` behind them, so it overlaps
 * the caller's next frame on `stream`.  `out` holds the frame once
 * `copy_stream` has reached that point (cudaStreamSynchronize or an event);
 * the caller keeps `out` alive and untouched until then.  The library writes
 * the frame into one of two device frames used in turn; `stream` waits for
 * the copy that read the same device frame two calls earlier.  Host
 * synchronisation and dropped frames as for dl_render_frame with a device
 * `out` (a dropped frame's copy delivers the device frame's earlier
 * contents).  DL_ERR_INVALID_ARG when `copy_stream` equals `stream` or a
 * pointer is NULL.
 */
dl_status dl_render_frame_async_host(dl_ctx* ctx, int32_t scene_id, int32_t display_id,
                                     const double L0_c2w[16], int32_t mode, float* out,
                                     void* stream, void* copy_stream);

/* Encoded image from per-ray colours (Sec. 4 step (3) and Sec. 6: the rays
 * of U_rays are rendered by any renderer, then the subpixels take their
 * channel by the precomputed ray indices): out[i] = ray_rgb[3 ray_of[i] +
 * (i mod 3)] for the 3wh subpixels i = (x*w + y)*3 + k.  ray_rgb: device,
 * N_rays x 3 FP32 (RGB of ray r, rays numbered as dl_get_ray_table reports
 * them); out: device, h x w x 3 FP32 (caller-owned).  Enqueued on `stream`;
 * NULL pointers are DL_ERR_INVALID_ARG. */
dl_status dl_encode_rays(dl_ctx* ctx, int32_t display_id, const float* ray_rgb, float* out,
                         void* stream);

/* Device bytes the last frame of (scene, display, mode) used for scratch,
 * or an estimate before any frame was rendered. */
dl_status dl_query_footprint(dl_ctx* ctx, int32_t scene_id, int32_t display_id, int32_t mode,
                             size_t* bytes);

/* Compositing tile shape of a mode (powers of two, 8..256 pixels each
 * side).  Defaults: DL_STANDARD 16x16, DL_DIRECTL and DL_REQUIRED_ONLY 32x32. */
dl_status dl_set_tile(dl_ctx* ctx, int32_t mode, int32_t tile_w, int32_t tile_h);

/*
 * Ray table without allocating (the paper has no counterpart: this serves
 * callers that cannot call cudaMalloc, such as code running inside another
 * library's memory pool, a process whose device memory is reserved up front,
 * or a real-time loop that must not synchronise the device the way
 * cudaMalloc/cudaFree can).  Builds the same table as dl_set_display /
 * dl_get_ray_table from a view map V (h*3w uint16) and subpixel map src
 * (3wh uint32) held in DEVICE memory, e.g. as returned by dl_get_view_map
 * and dl_get_subpixel_map with out_on_device = 1.  Writes ray_of (3wh
 * uint32, device) and rays ((view, row, col) int32 triplets, device, room
 * for 3*3wh entries; the first 3*N_rays are written), and *n_rays (host).
 * Needs no context and allocates nothing: its scratch is one file-scope
 * device array of 6.5 MiB that every GPU loading the library keeps until
 * exit, so panels are limited to width*height <= 65536 pixels (e.g. 256x256);
 * larger panels, NULL pointers or non-positive sizes return
 * DL_ERR_INVALID_ARG.  The first call on a device, with that device
 * current, looks the array's device address up and keeps it for the
 * process: a cudaDeviceReset on that device invalidates it, so the call must
 * not be used after one.  Enqueued on `stream`, then synchronises it once to
 * read the ray count.  All calls share the array, which keeps the last
 * call's contents:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and must be serialised by the caller.
 */
dl_status dl_ray_table_static(int32_t width, int32_t height, const uint16_t* V,
                              const uint32_t* src, uint32_t* ray_of, int32_t* rays,
                              int64_t* n_rays, void* stream);

/* Options of a context (dl_set_option).
 * DL_OPT_SORT_MODE: how each (view, tile) list of Gaussians gets its depth
 *   order.  DL_SORT_AUTO (default): keys are binned straight into their tile
 *   and every compositing block sorts its own list in shared memory, unless a
 *   list is longer than 16384 keys, in which case the frame uses one global
 *   stable LSD radix sort of (view, tile, depth) keys.  DL_SORT_RADIX: always
 *   the global radix sort.  DL_SORT_BINNED: always binned; a frame with a
 *   longer list fails with DL_ERR_CAPACITY.  Both give the same image. */
enum { DL_OPT_SORT_MODE = 1, DL_OPT_EVAL_DIRECTL = 2, DL_OPT_EVAL_STANDARD = 3,
       DL_OPT_WARP_LIST_CAP = 4, DL_OPT_STANDARD_VIEW_SIZE = 5, DL_OPT_HEAP_CAPACITY = 6,
       DL_OPT_KEY_EMISSION = 7 };
/* DL_OPT_KEY_EMISSION: where the binned path of DL_DIRECTL / DL_REQUIRED_ONLY
 * writes its tile keys, once a frame of the same signature has been sized.
 * 1: the projection kernel emits every (view, tile, Gaussian) key itself,
 * into per-(view, tile) slices of the key buffer laid out from the
 * signature's previous frame (its key count per group plus an eighth and
 * 16); a frame whose counts outgrow a slice emits its keys a second time
 * into slices sized from its own counts, on the device, before compositing.
 * 0: the projection writes per-(view, Gaussian) tile metadata and a second
 * kernel emits the keys into slices sized from this frame's counts (Sec. 4
 * step (2) as two passes).  2 (default): 1 for scenes of at least 131,072
 * Gaussians, else 0 (a small scene has too few warps in flight to hide the
 * projection's waits on its cursor atomics).  All give the same keys, so
 * the same image. */
/* DL_OPT_HEAP_CAPACITY: c_h of DL_RAYCAST, the number of nearest
 * intersections each ray keeps and blends (1..256, default 128).
 *
 * DL_RAYCAST: per ray (origin at its view's camera, unit direction d through
 * its pixel), every Gaussian with alpha_j = o_j G(o + t_j d) >= 1/255 at its
 * highest-density point t_j = (mu - o)^T S^-1 d / (d^T S^-1 d) > 0.2 (Eqs.
 * (16)-(17)) enters a max-heap that keeps the c_h smallest (t, index); they
 * are blended in t order (alpha clamped to 0.99, stop before T < 1e-4) with
 * the SH colour at d.  An 8-wide tree of the Gaussians' alpha >= 1/255
 * boxes (binary SAH splits over the scene's stored Morton order, collapsed
 * into 8-wide nodes; Sec. 7) is built on the GPU on the first such frame of
 * a scene and kept with it. */
/* DL_OPT_STANDARD_VIEW_SIZE: resolution at which DL_STANDARD renders each
 * view, value = (view_w << 16) | view_h, 0 = the panel's (HR).  Below panel
 * resolution (the LR / MR configurations of the paper's experiments) every
 * view is rendered at view_w x view_h with the same field of view, then
 * upsampled while interweaving (Alg. 1, "Resize ... Upsample"): subpixel
 * (x, y, k) takes channel k of its view V(x, 3y + k) bilinearly at
 * (y view_w / w, x view_h / h) of that view, clamped at the border.
 * 1 <= view_w, view_h <= 16384. */
enum { DL_SORT_AUTO = 0, DL_SORT_RADIX = 1, DL_SORT_BINNED = 2 };
/* DL_OPT_EVAL_DIRECTL / DL_OPT_EVAL_STANDARD: how a warp evaluates a tile's
 * Gaussians on the binned path.  DL_EVAL_DIRECT: every lane walks the
 * culled list for its own ray.  DL_EVAL_TRANSPOSED: each lane holds one
 * Gaussian and tests it against all of the warp's unfinished rays, then each
 * lane blends its own candidates in order.  Defaults: transposed for
 * DL_DIRECTL and DL_REQUIRED_ONLY, direct for DL_STANDARD.  Same image
 * either way. */
enum { DL_EVAL_DIRECT = 0, DL_EVAL_TRANSPOSED = 1 };
/* DL_OPT_WARP_LIST_CAP: on the binned DL_DIRECTL / DL_REQUIRED_ONLY path,
 * tile lists of up to this many keys (512 or 1024) are composited by one warp
 * each; longer lists by a thread block.  0 sends every list to thread
 * blocks.  Default 512.  Same image either way. */
dl_status dl_set_option(dl_ctx* ctx, int32_t option, int64_t value);

/* Statistics of frames rendered on the context. */
typedef struct {
    int64_t n_keys;          /* (view, tile, Gaussian) overlaps sorted        */
    int64_t n_rays;          /* rays composited (w*h*N_v for DL_STANDARD)    */
    int64_t pairs_evaluated; /* (ray, Gaussian) alpha evaluations, when
                                stage timing is on                           */
    int64_t pairs_blended;   /* of those, the ones composited (Eq. (5))      */
    int32_t tile_w, tile_h;
    int32_t sort_bits;       /* key bits the radix sort ordered              */
    int32_t n_launches;      /* kernels the frame launched                   */
    int64_t lists_small;     /* tile lists composited by the small class     */
    int64_t lists_large;     /* tile lists composited by the large class     */
    int64_t max_list;        /* longest tile list (keys)                     */
    int64_t n_visible;       /* (view, Gaussian) records the projection wrote
                                (in front of the near plane, alpha can reach
                                1/255 inside the view)                       */
    float ms_project, ms_scan, ms_sync, ms_emit, ms_sort, ms_ranges, ms_composite,
        ms_interweave, ms_total; /* stage durations (CUDA events)        */
    int32_t status;          /* last frame: 0 when complete, else the frame was
                                dropped (output left untouched): bit 0 its tile
                                keys exceeded the key capacity, bit 1 a tile
                                list exceeded the long-list capacity.  In
                                dl_stage_totals: the number of dropped frames */
    int32_t reemitted;       /* last frame: 1 when its keys outgrew the slices
                                its signature's previous frame laid out and the
                                projection emitted them again (key emission in
                                the projection, DL_OPT_KEY_EMISSION 1), else 0.
                                In dl_stage_totals: the number of such frames */
} dl_frame_stats;

/* While enabled, every dl_render_frame records CUDA events around its
 * stages on its stream, without synchronising.  enable = 1 also counts the
 * compositing pairs (pairs_evaluated / pairs_blended; the compositing kernels
 * then run their counting variant), enable = 2 records the events only,
 * enable = 0 turns both off (the default). */
dl_status dl_enable_stage_timing(dl_ctx* ctx, int32_t enable);
/* Counters of the last frame (stage times are 0: see dl_stage_totals);
 * waits for the last frame when its counters are still on the device. */
dl_status dl_last_frame_stats(dl_ctx* ctx, dl_frame_stats* out);
/* Sums of every field over the frames rendered with stage timing on since
 * the previous call (waits for those frames to finish), and their number.
 * tile_w/tile_h/sort_bits are those of the last frame. */
dl_status dl_stage_totals(dl_ctx* ctx, dl_frame_stats* sum, int32_t* n_frames);

/* ---- Frame batches ---------------------------------------------------
 * The paper renders one light-field frame at a time; it has no counterpart
 * for this section, which serves many DirectL frames (any mix of scenes,
 * displays, view counts and tile shapes) at once.
 *
 * A batch owns n_slots frame slots with fixed device capacities.  Every
 * dl_batch_launch renders one DirectL frame (the frame of Sec. 5, the same
 * image dl_render_frame gives) for each assigned slot without any host
 * synchronisation: per slot the projection, group scan, key emission and
 * list partition; then one persistent launch per compositing class over the
 * tile lists of all slots together; then each slot's reorder into the
 * caller's output.  So the sequence can be captured into a CUDA graph
 * (dl_batch_capture) and replayed.
 *
 * Capacities of slot i come from plans[i]: that frame is rendered once
 * through dl_render_frame (DL_DIRECTL, on `stream`, synchronously); its key
 * count times `margin` (>= 1) is the slot's key capacity and its longest
 * tile list times margin, rounded up to a power of two (2048..16384), the
 * batch's long-list capacity.  Its views x Gaussians, (view, tile) groups,
 * rays, tile lists and views are the slot's hard limits.  A launched frame
 * whose keys exceed the key capacity, or that has a tile list longer than
 * the long-list capacity, is not composited (its output is left as it was)
 * and is reported by dl_batch_wait.
 *
 * Ownership and lifetime: the library owns the batch's memory; the caller
 * owns each slot's output (device, h*w*3 FP32, the layout of
 * dl_render_frame) and must keep it valid while launches that write it are
 * in flight.  Assigned scenes and displays cannot be freed (DL_ERR_INVALID_ARG)
 * and the context cannot be destroyed while a batch exists.  Calls on one
 * batch are not thread-safe; the context's other calls may not run
 * concurrently with them either.  dl_batch_assign, dl_batch_clear and
 * dl_batch_set_pose wait for the batch's previous launch to finish (they
 * rewrite the host staging that the launch uploads). */
typedef struct dl_batch dl_batch;
typedef struct {
    int32_t scene_id, display_id;
    int32_t tile_w, tile_h;  /* 0, 0: the context's DL_DIRECTL tile            */
    double L0_c2w[16];       /* pose of the sizing frame (row-major 4x4)      */
} dl_slot_plan;
dl_status dl_batch_create(dl_ctx* ctx, int32_t n_slots, const dl_slot_plan* plans, double margin,
                          void* stream, dl_batch** out);
dl_status dl_batch_destroy(dl_batch* b);
/* Assigns a frame to a slot.  tile_w, tile_h as in dl_slot_plan.
 * DL_ERR_CAPACITY when the frame exceeds the slot's hard limits. */
dl_status dl_batch_assign(dl_batch* b, int32_t slot, int32_t scene_id, int32_t display_id,
                          int32_t tile_w, int32_t tile_h, float* out_dev);
dl_status dl_batch_clear(dl_batch* b, int32_t slot);
/* Light-field centre pose of the slot's next frame (row-major 4x4 c2w). */
dl_status dl_batch_set_pose(dl_batch* b, int32_t slot, const double L0_c2w[16]);
/* Enqueues one frame for every assigned slot on `stream`; replays the
 * captured graph when the assignment has not changed since the capture. */
dl_status dl_batch_launch(dl_batch* b, void* stream);
/* Captures the launch sequence of the current assignment into a CUDA graph
 * (stream capture on `stream`, which must not be the legacy default stream);
 * nothing runs during the capture.  Any assignment change drops the graph. */
dl_status dl_batch_capture(dl_batch* b, void* stream);
/* Waits for the last launch.  status (optional, n_slots entries): 0 ok, bit 0
 * key capacity exceeded, bit 1 a tile list longer than the long-list
 * capacity (only for assigned slots).  Returns DL_ERR_CAPACITY when a slot
 * failed. */
dl_status dl_batch_wait(dl_batch* b, uint32_t* status);
/* Device bytes the batch holds, and its long-list capacity. */
dl_status dl_batch_info(dl_batch* b, size_t* bytes, int32_t* long_list_cap);

/* Tile-shape autotuner (no counterpart in the paper): renders the DirectL
 * frame of (scene, display, pose) with each candidate tile shape
 * (n_candidates pairs {tile_w, tile_h} in `candidates`; powers of two,
 * 8..256), `reps` timed frames each after one warm-up frame, on `stream`,
 * and sets the context's DL_DIRECTL tile to the one with the lowest median
 * device time.  best[2] receives it; ms (optional, n_candidates entries) the
 * medians. */
dl_status dl_autotune_tile(dl_ctx* ctx, int32_t scene_id, int32_t display_id,
                           const double L0_c2w[16], const int32_t* candidates, int32_t n_candidates,
                           int32_t reps, void* stream, int32_t* best, float* ms);

/* Arithmetic peaks of `device` measured by microbenchmarks (no counterpart
 * in the paper; the benchmark's compositing roofline divides by them): FP32
 * fused multiply-adds as scalar and as packed FP32x2 instructions (TFLOP/s,
 * 2 FLOP per FMA) and ex2.approx results per second, each the best of three
 * timed launches that fill every SM.  Synchronous; allocates 1 KB of device
 * memory and one stream for the call. */
dl_status dl_measure_peaks(int32_t device, double* fp32_tflops, double* fp32x2_tflops,
                           double* ex2_per_s);

#ifdef __cplusplus
}
#endif
#endif
