/*
 * seele.h -- C ABI of the GB300 (sm_103a) implementation of the Seele
 * rendering hot path (arxiv 2503.05168, "Seele: A Unified Acceleration
 * Framework for Real-Time Gaussian Splatting on Mobile Devices").
 *
 * The library renders a set of 3D Gaussians (Sec. 3.1: centroid, covariance
 * from scale and rotation, opacity, spherical-harmonic colour) tile by tile
 * in three steps -- preprocessing, sorting, rasterization (Sec. 3.1) -- with
 * the paper's two techniques as options: hybrid preprocessing (Sec. 3.3:
 * view-cluster filter plus the opacity-aware online filter of Eqns. 3-5) and
 * contribution-aware rasterization (Sec. 3.4, Algorithm 1).  It also
 * differentiates the render for the fine-tuning of Sec. 3.5.
 *
 * Conventions shared by every call:
 *   - No C++ exception crosses this boundary; every call returns a status.
 *     On failure seele_last_error() describes the cause.
 *   - All GPU work is enqueued on the context's stream (borrowed, never
 *     destroyed by the library).  Pointers documented as "device" must be
 *     device (or managed) memory of the context's device; "host or device"
 *     pointers are classified with cudaPointerGetAttributes.
 *   - Float tensors are float32, row-major, tightly packed.
 *   - A context is not thread-safe: one host thread at a time.
 *
 * Scene layout (per Gaussian g, n Gaussians):
 *   means[g*3 + i]            world position, i = x, y, z
 *   log_scales[g*3 + i]       log of the per-axis standard deviation
 *   quats[g*4 + i]            rotation quaternion (w, x, y, z), any norm > 0
 *   opacity_logits[g]         opacity o = sigmoid(logit)
 *   sh[(g*nc + k)*3 + c]      SH coefficient k = l*l + l + m (real basis,
 *                             Condon-Shortley phase) of channel c,
 *                             nc = (sh_degree + 1)^2
 *   cluster_mask[g]           bit c set: g belongs to view cluster c; shared
 *                             Gaussians carry every bit (Sec. 3.3)
 *
 * Camera model: x right, y down, z forward; X_cam = R x + t with
 * world_to_cam = [R | t] row-major; u = fx X/Z + cx, v = fy Y/Z + cy in
 * continuous pixel units; pixel (px, py) is sampled at (px + .5, py + .5).
 * Output images are planar: for camera j, rgb[off_j*3 + c*H*W + y*W + x] and
 * T[off_j + y*W + x] with off_j = sum_{i<j} W_i*H_i.
 */
#ifndef SEELE_H
#define SEELE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct seele_ctx seele_ctx;

typedef enum {
    SEELE_OK = 0,
    SEELE_ERR_ARG = 1,       /* invalid argument (null pointer, size, option) */
    SEELE_ERR_STATE = 2,     /* call out of order (no scene, no cameras, no render) */
    SEELE_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    SEELE_ERR_CAPACITY = 4,  /* tile-instance capacity exceeded (async mode only) */
    SEELE_ERR_TIMEOUT = 5,   /* a bounded device spin-wait gave up */
    SEELE_ERR_OOM = 6,       /* device allocation failed */
    SEELE_ERR_INTERNAL = 7   /* a device consistency check failed (outputs undefined) */
} seele_status;

enum { SEELE_SCENE_COPY = 0, SEELE_SCENE_BORROW = 1, SEELE_SCENE_SPATIAL = 2 };

/* Scene description.  COPY: the library copies the attributes (host or device
 * pointers) into its own layout and owns that copy.  BORROW: the pointers are
 * device memory owned by the caller, must stay valid and unchanged in size
 * until the next seele_load_scene or seele_destroy, and are re-read by every
 * render (their contents may change between renders, as in training) and by
 * seele_render_backward, which needs them as the render it differentiates
 * read them.  When quats and sh are 16-byte aligned the kernels read the
 * arrays in place; otherwise every render first repacks them into the
 * library's layout.
 * COPY reads device and page-locked host arrays (cudaMallocHost,
 * cudaHostRegister) in place, the latter over the host link in the same pass
 * that repacks them; other host arrays are first copied to a device staging
 * area.
 * COPY | SPATIAL also stores the Gaussians in Morton order of their means
 * (computed on the device at load), so that Gaussians culled together are
 * stored together and preprocessing reads less of the scene.  Images are the
 * same up to Gaussians at exactly equal depth (ties break by stored index);
 * gradients and view-builder masks come back in the caller's order, while
 * record ids in seele_debug_view follow the stored order (its scene_order maps
 * them back). */
typedef struct {
    int64_t n;                    /* number of Gaussians, 1 <= n <= 16776960, n * cameras < 2^31 */
    int32_t sh_degree;            /* 0..3 */
    int32_t flags;                /* SEELE_SCENE_COPY or SEELE_SCENE_BORROW, optionally | SEELE_SCENE_SPATIAL */
    const float* means;           /* [n][3] */
    const float* log_scales;      /* [n][3] */
    const float* quats;           /* [n][4] */
    const float* opacity_logits;  /* [n] */
    const float* sh;              /* [n][(sh_degree+1)^2][3] */
    const uint32_t* cluster_mask; /* [n] or NULL (no view clusters) */
    int32_t n_clusters;           /* 0..32; centroids required if > 0 */
    float pos_scale;              /* position normalisation s of the cluster features */
    const float* centroids;       /* host, [n_clusters][6] = (x / s, view dir) */
} seele_scene_desc;

/* One camera (Sec. 3.1: a render takes a camera pose and viewing direction). */
typedef struct {
    float world_to_cam[12];       /* [R | t], row-major 3x4 */
    float fx, fy, cx, cy;         /* pinhole intrinsics, pixels */
    int32_t width, height;        /* 1..16384 */
    float near_z;                 /* Gaussians with Z <= near_z are culled (0.2) */
} seele_camera;

enum { SEELE_MODE_PLAIN = 0, SEELE_MODE_CR = 1 };

/* Tile test: which tiles of a Gaussian's bounding rect get an instance.
 * RECT keeps every tile of the rect of Sec. 3.3's support radius; ELLIPSE
 * keeps only the tiles whose pixel centres the support ellipse q <= t_g
 * reaches (inflated by 0.1% and widened by 1/256 px, so that no blended pixel
 * is lost to FP32 rounding).  Both give the same image; ELLIPSE has fewer
 * instances to sort and to rasterize. */
enum { SEELE_TILES_RECT = 0, SEELE_TILES_ELLIPSE = 1 };

/* Binning: the unit the sorted instance lists are kept per.
 * TILES: one (tile, Gaussian) instance per tile, sorted by tile after the
 * depth sort (Sec. 3.1).  BLOCKS: one instance per 8x4-tile block, carrying
 * a 32-bit mask of the block's tiles that the Gaussian reaches (same tile
 * test), sorted by block; each tile's rasterizer walks its block's list and
 * keeps the entries with its bit -- its tile list, in the same order.  Both
 * give the same image and per-pixel list positions; BLOCKS sorts several
 * times fewer instances and reads only the part of each list it rasterizes.
 * A backward pass after a BLOCKS render first re-bins the frame by tiles. */
enum { SEELE_BIN_TILES = 0, SEELE_BIN_BLOCKS = 1 };

/* Rasterizer schedule (not in the paper: how many cameras' tiles share the
 * GPU).  GRID: one CTA per list unit, launched longest lists first.  QUEUE:
 * one resident wave of CTAs that pull units from an atomic queue; the queue
 * takes the cameras in groups of batch_depth (the cameras with the least
 * rasterization work first: list lengths times the tiles that walk them),
 * each group's units longest lists first, so that the views of
 * an early group are finished before the next group starts -- per-view
 * latency falls while each group still balances its own tiles.  batch_depth
 * 0 puts every camera in one group (then QUEUE orders like GRID). */
enum { SEELE_SCHEDULE_GRID = 0, SEELE_SCHEDULE_QUEUE = 1 };

/* Render flags */
enum {
    SEELE_RENDER_ASYNC = 1,       /* do not synchronise; see seele_render */
    SEELE_RENDER_PROFILE = 2,     /* time each stage with CUDA events into seele_stats.stage_ms
                                     (synchronous renders only) */
    SEELE_RENDER_COUNT = 4,       /* count the rasterizer's work into seele_stats (slower
                                     variant; synchronous renders only) */
    SEELE_RENDER_GRAPH = 8        /* capture the frame into a CUDA graph on first use and
                                     replay it while the camera count and resolutions, the
                                     options, the instance capacity, the scene and the
                                     output pointers stay the same; camera poses may change
                                     between replays.  Device or page-locked host outputs */
};

/* Stages timed by SEELE_RENDER_PROFILE, in launch order. */
enum {
    SEELE_STAGE_PREPROCESS = 0,   /* scene repack (BORROW) + per-(camera, Gaussian) preprocessing */
    SEELE_STAGE_COMPACT = 1,      /* visible-record compaction */
    SEELE_STAGE_DEPTH_SORT = 2,   /* histogram + 4 radix passes on fp32 depth */
    SEELE_STAGE_TILE_SCAN = 3,    /* instance offsets in depth order */
    SEELE_STAGE_EMIT = 4,         /* tile instances */
    SEELE_STAGE_TILE_SORT = 5,    /* histogram + radix passes on the tile id */
    SEELE_STAGE_RANGES = 6,       /* per-tile list ranges */
    SEELE_STAGE_RASTER = 7,       /* blending (Eqns. 1-2 / Alg. 1) */
    SEELE_NUM_STAGES = 8
};

/* Render options.  seele_default_options fills the paper's constants. */
typedef struct {
    int32_t mode;                 /* PLAIN (Sec. 3.1) or CR (Alg. 1) */
    int32_t group_w, group_h;     /* CR pixel group: 2x2 (default), 1x1, 2x4, 4x4, 4x8 */
    int32_t tile_w, tile_h;       /* 16x16 (default), 32x8, 32x16 or 8x8 */
    int32_t opacity_filter;       /* 1: support min(2 ln(o/alpha_theta), 9) (Eqn. 5) */
    int32_t cluster_filter;       /* 1: render only the selected view clusters (Sec. 3.3) */
    int32_t n_neighbors;          /* M of Sec. 3.3 (3) */
    float alpha_min;              /* alpha_theta, 1/255 */
    float alpha_max;              /* alpha clamp, 0.99 */
    float t_stop;                 /* Gamma_theta, 1e-4 */
    int32_t flags;                /* SEELE_RENDER_* */
    int32_t tile_test;            /* SEELE_TILES_ELLIPSE (default) or SEELE_TILES_RECT */
    int32_t binning;              /* SEELE_BIN_BLOCKS (default) or SEELE_BIN_TILES */
    int32_t schedule;             /* SEELE_SCHEDULE_GRID (default) or SEELE_SCHEDULE_QUEUE */
    int32_t batch_depth;          /* QUEUE: cameras per group, 0 = all (default) */
} seele_options;

/* Per-render statistics (all cameras of the call). */
typedef struct {
    int64_t n_visible;            /* (camera, Gaussian) pairs that reach binning */
    int64_t n_instances;          /* sorted instances: (tile, Gaussian) pairs K, or
                                     (tile block, Gaussian) pairs with SEELE_BIN_BLOCKS */
    int64_t capacity;             /* instance capacity after the call */
    int32_t retries;              /* renders repeated after a capacity growth */
    int32_t n_kernels;            /* kernel launches of the last attempt */
    float stage_ms[8];            /* SEELE_RENDER_PROFILE: device time per stage, else 0 */
    int64_t leader_tests;         /* SEELE_RENDER_COUNT: Alg. 1 leader tests (CR only) */
    int64_t pairs_evaluated;      /* SEELE_RENDER_COUNT: (pixel, Gaussian) alphas evaluated */
    int64_t pairs_blended;        /* SEELE_RENDER_COUNT: pairs accumulated into the pixel */
} seele_stats;

/* Gradients, caller-owned device buffers in the scene layout; overwritten. */
typedef struct {
    float* means;                 /* [n][3] */
    float* log_scales;            /* [n][3] */
    float* quats;                 /* [n][4] */
    float* opacity_logits;        /* [n] */
    float* sh;                    /* [n][nc][3] */
} seele_grads;

/* Fills *opt with: PLAIN, 2x2 group, 16x16 tiles, filters off, M = 3,
 * alpha_theta = 1/255 (Sec. 3.1), clamp 0.99, Gamma_theta = 1e-4, flags 0,
 * ellipse tile test, block binning, grid schedule. */
void seele_default_options(seele_options* opt);

/* Creates a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the context,
 * owned by the caller and released with seele_destroy.  (The paper's renderer
 * state: the trained model and the per-frame buffers of Sec. 3.1's three
 * steps live in the context.)  Errors: SEELE_ERR_ARG for a NULL out or a
 * device that does not exist (no device at all included). */
seele_status seele_create(seele_ctx** out, int device, void* cuda_stream);

/* Releases every device buffer of the context.  NULL is ignored. */
void seele_destroy(seele_ctx* ctx);

/* Replaces the stream used by subsequent calls (borrowed). */
seele_status seele_set_stream(seele_ctx* ctx, void* cuda_stream);

/* Loads (COPY) or references (BORROW) a scene; see seele_scene_desc.
 * Invalidates any previous render state. */
seele_status seele_load_scene(seele_ctx* ctx, const seele_scene_desc* scene);

/* Streamed scene (Sec. 3.3 "Scene Prefetching").  Like seele_load_scene
 * (COPY, host memory only) with view clusters, but the device holds only the
 * shared Gaussians (mask with every cluster bit) and n_slots (1..64) slots of
 * slot_gaussians Gaussians (0: the largest cluster's size); every cluster's
 * Gaussians stay in pinned host memory (a Gaussian of several clusters is
 * copied into each), cut into chunks of at most slot_gaussians, one per slot.
 * Renders need the cluster filter, and the chunks of the clusters a frame's
 * cameras select must fit the slots.  Before a frame, those chunks are loaded
 * into slots on the render stream if not resident (the least recently used
 * slot is refilled); a Gaussian held by several selected
 * clusters' slots is drawn from the lowest cluster's, so the frame renders the
 * same Gaussians as the whole scene with the cluster filter.  After a frame,
 * each camera's position and viewing direction are extrapolated linearly
 * `ahead` (>= 1) frames from its last two frames, and the clusters selected
 * for that pose are prefetched (their chunks) into slots the frame does not read, on a
 * separate copy stream that waits only for the last frame reading the slot;
 * the next frame waits for a prefetched slot only when it needs it.
 * Gradients, the view builder and the skew statistic need seele_load_scene. */
seele_status seele_load_scene_streamed(seele_ctx* ctx, const seele_scene_desc* scene, int32_t n_slots,
                                       int64_t slot_gaussians, int32_t ahead);

/* Makes dst render the scene src holds, without a copy: dst keeps its own
 * stream, cameras, frame workspace and captured graph, so frames of the two
 * contexts may be in flight at once on their streams (one frame's
 * rasterization overlapping the next frame's preprocessing and sorting).
 * The device memory of a COPY scene is reference counted: it stays valid
 * until every context sharing it has loaded another scene or been destroyed,
 * so either context may later reload or be destroyed; the others keep
 * rendering the scene as it was shared.  A BORROW scene is referenced by dst
 * as by src (the caller keeps its arrays alive and unchanged); dst repacks
 * it into its own planes each frame.  View clusters, the spatial order and
 * the cluster mask come along; every call that reads the scene works on dst,
 * and none writes it.
 *   dst, src  contexts on the same device; src holds a scene loaded by
 *             seele_load_scene (or shared into it); dst may hold any state,
 *             which is dropped as by seele_load_scene.
 * Errors: SEELE_ERR_ARG for NULL, dst == src or different devices;
 * SEELE_ERR_STATE when src has no scene or a streamed one (its slots change
 * every frame).  Contexts sharing a scene may be used from different host
 * threads; loading, sharing and destroying contexts are not thread safe
 * with respect to each other. */
seele_status seele_share_scene(seele_ctx* dst, const seele_ctx* src);

typedef struct {
    int64_t resident_bytes;    /* device bytes of the resident Gaussians (attributes and masks) */
    int64_t full_bytes;        /* the same for the whole scene resident */
    int64_t n_shared;          /* resident shared Gaussians */
    int64_t slot_capacity;     /* Gaussians per slot */
    int64_t n_slots;
    int64_t n_chunks;          /* chunks the clusters are cut into */
    int64_t frames;            /* frames rendered since the load */
    int64_t loads_sync;        /* chunks a frame had to load itself */
    int64_t loads_prefetched;  /* chunks loaded ahead on the copy stream */
    int64_t prefetch_hits;     /* prefetched chunks a later frame used */
    int64_t resident_hits;     /* needed chunks already resident from earlier frames */
} seele_stream_stats;

seele_status seele_get_stream_stats(const seele_ctx* ctx, seele_stream_stats* out);

/* Sets n >= 1 cameras (host array, copied).  With view clusters loaded, also
 * runs the runtime cluster selection of Sec. 3.3 on the host: the nearest
 * centroid to the camera feature (position / s, view direction) and the
 * opt-independent M = n_neighbors(3) centroids nearest to it. */
seele_status seele_set_cameras(seele_ctx* ctx, const seele_camera* cams, int32_t n);

/* Renders every camera set by seele_set_cameras: Sec. 3.1's preprocessing,
 * sorting and tile rasterization (Eqns. 1-2), with the options' hybrid
 * preprocessing (Sec. 3.3, Eqns. 3-5) and contribution-aware rasterization
 * (Sec. 3.4, Algorithm 1).
 *   out_rgb  host or device, [sum_j 3 W_j H_j] planar per camera (see top)
 *   out_T    host, device or NULL, [sum_j W_j H_j] final transmittance
 *   stats    host or NULL
 * Without SEELE_RENDER_ASYNC the call synchronises the stream, grows the
 * instance capacity and re-renders when it was exceeded, and returns the
 * device status.  With SEELE_RENDER_ASYNC it returns after enqueueing; the
 * outputs must then be device or page-locked host memory, and a host output
 * is written by a copy enqueued after the frame on the same stream.  A
 * capacity overflow then leaves the outputs undefined and is reported by
 * seele_synchronize, after which the next render uses the grown capacity.
 * SEELE_RENDER_GRAPH takes the same outputs. */
seele_status seele_render(seele_ctx* ctx, const seele_options* opt, float* out_rgb, float* out_T,
                          seele_stats* stats);

/* Waits for the stream and returns the device status of the work enqueued
 * since the previous check (CAPACITY, TIMEOUT or OK). */
seele_status seele_synchronize(seele_ctx* ctx);

/* Gradient of sum(dL_drgb * rgb) for the last seele_render (same scene,
 * cameras and options; else SEELE_ERR_STATE), for the fine-tuning of
 * Sec. 3.5.  dL_drgb is device memory in
 * the out_rgb layout.  Skip and stop decisions of the forward pass are held
 * fixed (Sec. 3.5: hybrid preprocessing and the CR skips are left out of
 * the gradient);
 * per-pixel transmittance is recomputed back to front, not stored. */
seele_status seele_render_backward(seele_ctx* ctx, const float* dL_drgb, const seele_grads* grads);

/* Read-only views of the last render's intermediates (device pointers owned
 * by the context, valid until the next load/render).  For tests and tools. */
typedef struct {
    int64_t n_records;            /* cameras * n */
    int64_t n_visible;
    int64_t n_instances;
    int64_t n_tiles;              /* list units over all cameras: tiles, or tile blocks
                                     with SEELE_BIN_BLOCKS */
    const uint32_t* inst_record;  /* [n_instances] record id = camera * n + g, grouped by
                                     global unit, front to back within a unit */
    const uint32_t* tile_start;   /* [n_tiles]: unit t's list is inst_record[tile_start[t] ..
                                     tile_end[t]); a unit without instances has
                                     tile_start >= tile_end */
    const uint32_t* tile_end;     /* [n_tiles] */
    const uint32_t* tiles_touched;/* [n_records] 0 = culled */
    const float* records;         /* [n_records][16] raster record (64 bytes): u, v,
                                     -A/2*log2e, -B*log2e, -C/2*log2e (conic
                                     [[A,B],[B,C]] = Sigma'^-1), log2 o, e_thr,
                                     the tile test's bound on -(cA dx^2 + cB dx dy
                                     + cC dy^2), r, g, b, clamp flag (1 when
                                     log2 o is within 1e-4 of log2 of the alpha
                                     clamp, else 0), then the tile box as
                                     two uint32 x0 | y0 << 16, x1 | y1 << 16, 0, 0;
                                     a pixel at offset (dx, dy) takes the Gaussian
                                     iff e = cA dx^2 + cB dx dy + cC dy^2 + log2 o
                                     >= e_thr, with alpha = min(clamp, 2^e) */
    const float* depth;           /* [n_records] camera-space Z */
    const uint32_t* n_contrib;    /* [sum W*H] 1 + last blended position in the
                                     pixel's tile list */
    const uint32_t* inst_mask;    /* SEELE_BIN_BLOCKS: [n_instances] tiles of the block the
                                     entry reaches, bit j*8 + i for tile (i, j); else NULL */
    const uint32_t* scene_order;  /* SEELE_SCENE_SPATIAL: [n] the caller's index of stored
                                     Gaussian g (record id = camera * n + g); else NULL */
    const uint32_t* mask_summary; /* SEELE_BIN_BLOCKS: [ceil(n_instances / 32)] OR of the
                                     masks of inst_mask[32 g .. 32 g + 31] (entries below
                                     n_instances); else NULL */
} seele_debug_view;

seele_status seele_get_debug_view(const seele_ctx* ctx, seele_debug_view* out);

/* Per-view completion times of the last completed render: out_ms[j] = time
 * from the start of preprocessing to the moment the last tile of camera j
 * finished blending (device clock).  n must equal the camera count; waits for
 * the stream. */
seele_status seele_get_view_times(const seele_ctx* ctx, float* out_ms, int32_t n);

/* Chooses the tile shape (16x16, 32x8, 32x16 or 8x8; Sec. 3.1 renders
 * "tile by tile", the tile size is the renderer's choice) that renders the
 * current scene and cameras fastest with *inout's other options, by timing a few
 * renders of each; writes it into *inout and the time per render into
 * *best_ms (nullable).  Leaves no render state behind.  (Batched multi-view
 * frames are not in the paper; its renders are one camera at a time.) */
seele_status seele_autotune(seele_ctx* ctx, seele_options* inout, float* best_ms);

/* What seele_autotune_ex minimises over the renders it times. */
enum { SEELE_TUNE_BATCH_MS = 0, SEELE_TUNE_VIEW_P50 = 1, SEELE_TUNE_VIEW_P99 = 2 };

typedef struct {
    float batch_ms;               /* device time of one render of all cameras */
    float view_p50_ms;            /* per-view completion times (seele_get_view_times) over */
    float view_p99_ms;            /*   the cameras of the timed renders: median, 99th pct. */
    int32_t from_cache;           /* 1: the choice came from the cache, nothing was timed */
    int32_t candidates;           /* configurations timed */
} seele_tune_result;

/* The batched multi-view autotuner (not in the paper): tile shape, then
 * schedule and batch depth.  Stage 1 times the four tile shapes with the
 * GRID schedule (batch time); stage 2, with the best shape, times GRID and
 * QUEUE with batch_depth 0 and n/2, n/4, ... 1 (at most 8 depths) and keeps
 * the configuration with the least `objective`.  Each candidate: two
 * warm-up renders, five timed CUDA-graph renders (batch time), and the view
 * times of those renders.
 *   cache_path  NULL, or a JSON file of earlier choices keyed by the device
 *               (name, SM count), the scene size (ceil log2 n), the cameras'
 *               resolutions, the render options that shape the work and the
 *               objective; a hit is returned without timing, a miss is timed
 *               and written back (the file is replaced atomically).
 * Writes the choice into *inout (tile_w, tile_h, schedule, batch_depth) and
 * the measurements into *result (nullable).  Leaves no render state behind. */
seele_status seele_autotune_ex(seele_ctx* ctx, seele_options* inout, int32_t objective, const char* cache_path,
                               seele_tune_result* result);

/* Builds the offline view-dependent representation of the loaded scene
 * (Sec. 3.3 "Offline Clustering").
 *   poses        host, [n_poses] sampled cameras (any image sizes)
 *   n_clusters   N of Sec. 3.3, 1..32;  n_poses >= n_clusters
 *   top_k        k of Sec. 3.3 (32), 1..64
 *   uniforms     host, [n_clusters] draws in [0, 1) that drive k-means++
 *   max_iter     Lloyd updates at most (100)
 * Poses are clustered by k-means on the feature (x / s, v) -- camera centre
 * over s = the largest camera distance of the samples, and the unit viewing
 * direction (beta = 1): seeding picks point floor(u_0 n), then the first point
 * whose running sum of squared distances to the chosen centres exceeds
 * u_j times their total; Lloyd iterations assign to the nearest centre (ties
 * to the lower index) and move centres to the means, until nothing changes.
 * Every pose is then rendered plainly (t_g = 9, no filters) and, per pixel,
 * the k Gaussians with the largest contribution Gamma_i alpha_i (ties to the
 * lower index) are found; a Gaussian gets bit c of its mask when it is such a
 * contributor for some pose of cluster c.  Gaussians of every cluster are the
 * shared ones; a zero mask drops the Gaussian.
 *   out_centroids  host, [n_clusters][6] (the seele_scene_desc layout)
 *   out_pos_scale  host, s (the seele_scene_desc position scale)
 *   out_mask       host or device, [n] (the seele_scene_desc cluster mask)
 *   out_assign     host or NULL, [n_poses] cluster of each pose
 * Synchronous; leaves the context's cameras as they were and no render
 * state behind. */
seele_status seele_build_view_clusters(seele_ctx* ctx, const seele_camera* poses, int32_t n_poses,
                                       int32_t n_clusters, int32_t top_k, const double* uniforms,
                                       int32_t max_iter, float* out_centroids, float* out_pos_scale,
                                       uint32_t* out_mask, int32_t* out_assign);

/* Contribution skew of the current cameras (Sec. 1 "Rendering
 * Inefficiency", Sec. 3.4 "Motivation"): the cameras are rendered with the
 * plain rules (Sec. 3.1; no opacity or cluster filter, tile lists) and, per
 * pixel, the contributions Gamma_i alpha_i of the Gaussians it blends are
 * ranked in descending order.
 *   opt          tile size, tile test, alpha_min / alpha_max / t_stop (NULL:
 *                defaults); its mode, filters, binning and flags are ignored
 *   frac         the share of the pixel's total to reach, 0 < frac <= 1 (0.99)
 *   out_m        [sum W*H] smallest number of the largest contributions whose
 *                sum reaches frac of their total (ties at the cut all count;
 *                0 where nothing blends)
 *   out_blended  [sum W*H] number of contributions
 *   out_walked   [sum W*H] tile-list entries the pixel examined (up to and
 *                including the one that would have crossed t_stop, else all)
 *   out_total    [sum W*H] sum of the contributions (1 - final T)
 *   out_listed   [sum W*H] or NULL: length of the pixel's tile list
 * Outputs are host or device memory, each camera's pixels row-major after the
 * previous camera's.  Synchronous; leaves no render state behind. */
seele_status seele_contribution_skew(seele_ctx* ctx, const seele_options* opt, float frac, uint32_t* out_m,
                                     uint32_t* out_blended, uint32_t* out_walked, float* out_total,
                                     uint32_t* out_listed);


/* Message of the last failed call on this context (library-owned). */
const char* seele_last_error(const seele_ctx* ctx);

/* Measured issue rates of the pipes the blending runs on (Sec. 3.1 Eqns.
 * 1-2, Alg. 1), the denominators of its roofline: every SM of `device` is
 * filled with independent chains of one instruction kind and each rate is
 * lane-operations per second from CUDA-event times (best of 3, after a
 * warm-up), at whatever SM clock the device runs.  Takes a few milliseconds
 * per kernel on `cuda_stream`; allocates 256 bytes; synchronous.
 *   fp32: fused multiply-add (one op per FMA), sfu: ex2.approx, alu: float
 *   min/max and three-input integer logic. */
typedef struct {
    int32_t sm_count;             /* cudaDevAttrMultiProcessorCount */
    int32_t sm_clock_max_mhz;     /* cudaDevAttrClockRate / 1000 */
    double fp32_tops;             /* 1e12 lane-ops/s */
    double sfu_tops;
    double alu_fmnmx_tops;
    double alu_lop3_tops;
    float fp32_ms, sfu_ms, alu_fmnmx_ms, alu_lop3_ms;  /* timed launch of each */
} seele_peaks;

seele_status seele_measure_peaks(int device, void* cuda_stream, seele_peaks* out);

/* Exclusive prefix sum out[i] = in[0] + ... + in[i-1] (mod 2^32) by the
 * single-pass decoupled look-back scan that seele_sort_tile_instances_noalloc
 * runs, on caller memory, with a test hook for its bounded wait.  The paper
 * has no counterpart (a service of the library).
 *   in, out         device, [n]; in 16-byte aligned
 *   scratch         device, seele_scan_scratch_bytes(n) bytes, 256-byte
 *                   aligned, any contents (cleared by the call)
 *   withhold_block  test hook: the scan block that takes this ticket (blocks
 *                   of 4096 elements, in launch order) publishes nothing, so
 *                   its successor's wait runs out; UINT32_MAX for none
 *   spin_limit      polls of a predecessor before a waiting block gives up,
 *                   records a timeout and goes on as if that predecessor's
 *                   prefix were zero (0: the library's limit, about a second)
 * Returns after the stream has finished: SEELE_OK, SEELE_ERR_TIMEOUT when a
 * wait gave up (out is then wrong from that block on), SEELE_ERR_ARG for NULL
 * or misaligned pointers. */
size_t seele_scan_scratch_bytes(uint32_t n);
seele_status seele_exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, void* scratch,
                                  uint32_t withhold_block, uint32_t spin_limit, void* cuda_stream);

/* Sorting tile instances without allocating.  The paper has no counterpart:
 * this is a service of the library, not a step of the method.
 *
 * Sorts tile instances given in front-to-back order into per-tile lists, as
 * the render path does between emission and rasterization, for callers that
 * cannot call cudaMalloc: hosts that own the device memory budget and forbid
 * outside allocations, or real-time loops where an allocation (which can
 * synchronise the device) would stall a frame.  All scratch lives in one
 * file-scope device array of the library, reserved on every GPU that loads
 * it until the process exits (about 8.4 MB); nothing is allocated or freed.
 *
 *   inst_tile[i], inst_record[i]  device, [n_instances]: tile id (< n_tiles)
 *                                 and payload of instance i, in the order the
 *                                 lists must keep (stable); inst_tile must be
 *                                 16-byte aligned (it is read as vectors)
 *   sorted_record                 device, [n_instances]: payloads grouped by
 *                                 tile, in input order within a tile
 *   tile_start, tile_end          device, [n_tiles]: tile t's list is
 *                                 sorted_record[tile_start[t] .. tile_end[t]);
 *                                 an empty tile has tile_start >= tile_end
 *   cuda_stream                   the stream to run on (NULL: legacy default)
 * Limits: n_instances <= SEELE_NOALLOC_MAX_INSTANCES, 1 <= n_tiles <=
 * SEELE_NOALLOC_MAX_TILES; larger sizes, a NULL or misaligned pointer return
 * SEELE_ERR_ARG before any GPU work.  A tile id >= n_tiles is found on the
 * device: nothing is sorted, every list is left empty and the call returns
 * SEELE_ERR_ARG.  The call runs on the current CUDA device and returns after
 * the stream has finished the sort (SEELE_ERR_TIMEOUT if a bounded device
 * wait gave up, SEELE_ERR_INTERNAL for any other device error).  The first call on a device also looks up the array's device
 * address; make that first call before any stream capture.  Every call
 * shares the one array and it keeps the last call's contents: calls that
 * overlap on the GPU (other streams or threads) race on it. */
#define SEELE_NOALLOC_MAX_INSTANCES (1u << 20)
#define SEELE_NOALLOC_MAX_TILES (1u << 16)
seele_status seele_sort_tile_instances_noalloc(const uint32_t* inst_tile, const uint32_t* inst_record,
                                               uint32_t n_instances, uint32_t n_tiles, uint32_t* sorted_record,
                                               uint32_t* tile_start, uint32_t* tile_end, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SEELE_H */
