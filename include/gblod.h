/*
 * gblod.h -- C ABI of the GB300-native level-of-detail particle renderer.
 *
 * Method: Szalay, Springel & Lemson, "GPU-Based Interactive Visualization of Billion Point
 * Cosmological Simulations" (arXiv:0811.2055).  The paper's three requirements -- simplify
 * the data into visually equivalent levels of detail, index them spatially, and let the
 * renderer decide per view what to draw -- become two calls:
 *
 *   gblod_build_lod(particles, masses, n_max) -> octree      (octree paragraph)
 *   gblod_render(octree, camera, resolution)  -> image       (depth and GPU paragraphs)
 *
 * plus a brute-force render of every particle (the "full rendering" the LOD image must be
 * indistinguishable from, abstract).  Every computation runs in the library's sm_103a CUDA
 * kernels; this header has no CUDA or torch types.
 *
 * Conventions for every call below:
 *   - Pointers named d_* are device pointers (cudaMalloc / torch CUDA tensors) on the current
 *     CUDA device; h_* are host pointers.  Caller-owned buffers are only read or written by
 *     work enqueued on `stream` during the call, so they must stay valid until that work is
 *     done.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Arguments are checked on the host before anything is enqueued; on any error the
 *     out-parameters are left untouched and nothing has been written.
 *   - Device-side checks (fixed-point range) set a sticky status word in the renderer that
 *     gblod_renderer_status() returns; the device never traps or waits without a bound.
 *   - Errors: gblod_status codes; gblod_last_error() gives a message for the calling thread.
 */
#ifndef GBLOD_H
#define GBLOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBLOD_OK = 0,
    GBLOD_ERR_INVALID_ARG = 1,   /* a pointer, size or parameter is invalid */
    GBLOD_ERR_RANGE = 2,         /* a mass, or a fixed-point amplitude / sum, is out of range */
    GBLOD_ERR_OOM = 3,           /* the allocator returned NULL */
    GBLOD_ERR_CUDA = 4,          /* a CUDA runtime call failed (message in gblod_last_error) */
    GBLOD_ERR_DEVICE_TIMEOUT = 5,/* a bounded device wait ran out */
    GBLOD_ERR_NOT_IMPLEMENTED = 6,
    GBLOD_ERR_CAPACITY = 7       /* a batch needed more reserved scratch than it had; its images are invalid */
} gblod_status;

/* ----------------------------------------------------------------- memory */
/* Optional allocation hook (e.g. the torch caching allocator).  alloc returns device memory
 * usable on `stream` or NULL; free releases it after the work already enqueued on `stream`.
 * A NULL gblod_allocator* (or NULL alloc) selects, for builds and octrees, the library's own
 * stream-ordered memory pool of the current device (cudaMallocFromPoolAsync / cudaFreeAsync), and,
 * for renderers (grow-only buffers), cudaMallocAsync / cudaFreeAsync on the device's default pool.
 * The library's pool keeps the memory freed into it mapped, for the next builds (a build frees its
 * sort buffers before it allocates the sorted arrays; an octree's arrays return to it when freed):
 * it holds at most the builds' peak footprint.  gblod_trim_cache returns it. */
typedef void *(*gblod_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*gblod_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
typedef struct {
    gblod_alloc_fn alloc;
    gblod_free_fn free;
    void *ctx;
} gblod_allocator;

/* ----------------------------------------------------------------- octree */
#define GBLOD_NODE_LEAF 1u     /* stores its particles verbatim */
#define GBLOD_NODE_INTERNAL 2u /* has children */
#define GBLOD_NODE_LOSSY 4u    /* depth-21 node holding more than n_max particles */
#define GBLOD_NODE_REPS 8u     /* stores n_max representatives (INTERNAL or LOSSY) */
#define GBLOD_MAX_DEPTH 21

/* Octree build parameters (octree paragraph: "at most n points (in our case, n=16000)"). */
typedef struct {
    uint64_t seed;        /* keys the counter-based generator of the subselection */
    uint32_t n_max;       /* at most n_max points per node; >= 1 */
    uint32_t reserved;
    double root_lo[3];    /* root cube [root_lo, root_lo + root_side)^3; finite */
    double root_side;     /* > 0 and finite */
} gblod_build_params;

/* One node of the octree, breadth-first order (depth, then locational code).  112 bytes. */
typedef struct {
    uint64_t code;        /* locational code (1 << 3*depth) | octant path */
    uint64_t seg_first;   /* first position in the (key, id)-sorted particle order */
    uint64_t point_first; /* first stored point in the packed point arrays */
    uint64_t mass_lo;     /* exact node mass: sum of mass * 2^47, low 64 bits */
    uint64_t mass_hi;     /* ... high 64 bits */
    uint32_t seg_count;   /* particles inside the node */
    uint32_t point_count; /* stored points: seg_count for leaves, n_max otherwise */
    uint32_t child_first; /* index of the first child (0 if none) */
    uint32_t child_count; /* non-empty octants */
    int32_t depth;
    int32_t flags;        /* GBLOD_NODE_* */
    int32_t parent;       /* -1 for the root */
    int32_t pad;
    float h_cull;         /* largest smoothing length drawn anywhere in the subtree */
    float w_rep;          /* weight of each representative, fp32(M_node / n_max); 0 for leaves */
    float s_rep;          /* smoothing-length scale of the representatives; 1 for leaves */
    float pad2;
    float bmin[3];        /* bounds of the node's particles */
    float bmax[3];
} gblod_node;

typedef struct gblod_octree gblod_octree; /* opaque, device resident, library owned */

typedef struct {
    uint64_t n_particles;
    uint64_t n_nodes;
    uint64_t n_points;    /* stored points over all nodes */
    uint64_t device_bytes;
    int32_t depth_max;
    int32_t equal_mass;   /* 1 if every particle had the same mass (raw draws are the keys) */
    uint32_t n_max;
    uint32_t formats;     /* bit 0: fp32 points held; bit 1: 16-bit block codes held */
} gblod_octree_info;

/* Builds the octree on the device (octree paragraph; A1 Morton keys, A2 radix sort, A3 node
 * counting, A4 density-weighted subselection, A5 representatives).
 *   d_xyz   n x 3 float32 positions (row-major), d_mass n float32 in [2^-24, 2^24], d_h n
 *           float32 smoothing lengths; d_ids NULL (particle id = input index) or n distinct
 *           uint32 ids that key the generator (so a permutation of rows with their ids gives
 *           the same tree); n < 2^32.
 *   Memory for the octree comes from `alloc` (kept by the octree and used again to free it).
 *   The call synchronises `stream` a few times (the host needs the node counts) and returns
 *   when the octree is complete.  GBLOD_ERR_RANGE if a mass is outside [2^-24, 2^24] or not
 *   finite. */
gblod_status gblod_build_lod(const float *d_xyz, const float *d_mass, const float *d_h, const uint32_t *d_ids,
                             uint64_t n, const gblod_build_params *params, const gblod_allocator *alloc,
                             void *stream, gblod_octree **out);

/* Frees the octree (after work already enqueued on the build's allocator stream semantics:
 * the caller must make sure no render using it is still running). */
void gblod_octree_free(gblod_octree *octree);

gblod_status gblod_octree_get_info(const gblod_octree *octree, gblod_octree_info *out);

/* Copies octree arrays to host buffers (each may be NULL; sizes from gblod_octree_get_info):
 *   h_nodes n_nodes gblod_node; h_pts4 n_points x 4 float (x, y, z, weight); h_hs n_points
 *   float; h_pt_src n_points uint32 (sorted position each stored point copies); h_skey
 *   n_particles uint64 sorted Morton keys; h_sidx n_particles uint32 input index per sorted
 *   position.  Synchronous. */
gblod_status gblod_octree_export(const gblod_octree *octree, gblod_node *h_nodes, float *h_pts4, float *h_hs,
                                 uint32_t *h_pt_src, uint64_t *h_skey, uint32_t *h_sidx);

/* ----------------------------------------------------------------- 16-bit block codes */
/* Storage paragraph: positions are kept in 2 bytes per coordinate spanning the block (node)
 * that holds the point, and the other properties are coded the same way, which halves the
 * bytes read per drawn point (10 instead of 20).  Codes, per node i and stored point j:
 *   qa[i] = (qlo_x, qlo_y, qlo_z, qstep, w_lo, w_step, h_lo, h_step)  8 floats
 *     qlo = fp32(corner of the node's cell), qstep = fp32(edge 2^-16);
 *     w_lo / h_lo = smallest finite value among the node's points (+0 for a zero),
 *     *_step = fp32((largest - smallest) / 65535) computed in double (0 if none finite).
 *   position code c = floor(((double)x - qlo) / qstep) clamped to 0..65535, NaN -> 0;
 *     decoded x' = qlo + (c + 1/2) qstep   (fp32, each operation rounded to nearest, no FMA);
 *   w and h codes c = rne(((double)v - lo) / step) clamped to 0..65535 (0 when the step is 0
 *     or v is not finite); decoded v' = lo + c step  (fp32, no FMA).
 * A point inside its cell decodes within edge 2^-17 of itself (plus the final fp32 rounding);
 * a point outside the root cube (clamped into a boundary cell by the build) decodes inside the
 * cell.  The quantised node table is the octree's own with bmin / bmax / h_cull replaced by the
 * bounds and the largest decoded h of the decoded points of each subtree, so culling stays
 * conservative for what is drawn. */
#define GBLOD_POINTS_FLOAT 0   /* fp32 (x, y, z, w) + h: 20 bytes per point */
#define GBLOD_POINTS_BLOCK16 1 /* 16-bit block codes: 10 bytes per point (gblod_octree_quantize) */

#define GBLOD_QUANTIZE_DROP_FLOAT 1u /* free the fp32 points once coded (GBLOD_POINTS_FLOAT then fails) */

/* Codes every stored point of the octree on the device (enqueued on `stream`, which it then
 * synchronises) and keeps the codes with the octree.  Calling it again is a no-op apart from
 * `flags`.  GBLOD_ERR_INVALID_ARG if the fp32 points were already dropped and no codes exist. */
gblod_status gblod_octree_quantize(gblod_octree *octree, uint32_t flags, void *stream);

/* Copies the block codes to host buffers (each may be NULL): h_codes n_points x 5 uint16
 * (x, y, z, w, h); h_qa n_nodes x 8 float (see above); h_qnodes n_nodes gblod_node, the
 * quantised node table.  Synchronous.  GBLOD_ERR_INVALID_ARG if the octree holds no codes. */
gblod_status gblod_octree_export_block16(const gblod_octree *octree, uint16_t *h_codes, float *h_qa,
                                         gblod_node *h_qnodes);

/* ----------------------------------------------------------------- rendering */
/* Pinhole camera (depth paragraph; GPU paragraph).  right/up/fwd are orthonormal rows;
 * image coordinates: u = cx + f_px * x_c / z_c, v = cy - f_px * y_c / z_c (y points down);
 * points with z_c <= z_near are not drawn.  width, height in 1..16384. */
typedef struct {
    double eye[3], right[3], up[3], fwd[3];
    double f_px, cx, cy, z_near;
    int32_t width, height;
} gblod_camera;

#define GBLOD_KERNEL_GAUSSIAN 0 /* truncated at 3 sigma, sigma = h */
#define GBLOD_KERNEL_CUBIC 1    /* M4 cubic spline with support 2h (the paper's "radial cubic") */

typedef struct {
    double lambda_px;     /* detail threshold: refine while (f * edge)^2 > lambda^2 max(D^2, z_near^2);
                             negative selects the default sqrt(n_max) */
    double sigma_min_px;  /* blob size clamp in pixels, 0 < min <= max (default 0.5, 128) */
    double sigma_max_px;
    double tone_lo, tone_hi; /* fixed log range in intensity units (used when tone_auto == 0) */
    int32_t kernel;       /* GBLOD_KERNEL_* */
    int32_t tone_auto;    /* 1: hi = image maximum, lo = 1e-4 hi */
    int32_t tile_w, tile_h; /* screen tile, 1..64 each, covering at most 8 strips of 8 x 16
                             pixels (ceil(w/8) ceil(h/16) <= 8; 0 = 64 wide, 16 high); any value gives the
                             same image */
    uint64_t record_budget; /* most (tile, splat) records held at once (16 bytes each); 0 = 2^28,
                             capped at 2^31.  A frame needing more is binned and splatted in
                             several passes over ranges of its points, with the same image */
    int32_t point_format; /* GBLOD_POINTS_*: which stored form of the octree's points is drawn */
    int32_t flags;        /* GBLOD_RENDER_*: 0 or GBLOD_RENDER_COUNT_UPDATES */
} gblod_render_params;

/* Count the pixel updates of the splat ((splat, pixel) pairs inside the kernel support) into
 * gblod_frame_stats.pixel_updates.  Instrumentation only: it does not change the image, and the
 * splat kernel runs about 10% slower with it. */
#define GBLOD_RENDER_COUNT_UPDATES 1

/* Render workspace: scratch buffers (grown on demand through the allocator), the sticky
 * device status word and the last frame's counters.  One renderer must not be used by two
 * calls that overlap on the device. */
typedef struct gblod_renderer gblod_renderer;

gblod_status gblod_renderer_create(const gblod_allocator *alloc, gblod_renderer **out);
void gblod_renderer_destroy(gblod_renderer *r);

/* LOD frame (R1 node selection, R2 projection and binning, R3 tiled splat, R4 tone map).
 *   d_image  height x width uint8 (row-major) or NULL; d_accum height x width uint64
 *   fixed-point intensities (2^-32 units) or NULL (then an internal buffer is used).
 *   Enqueued on `stream`; the call waits once on `stream` mid-frame to size the splat lists.
 *   params->point_format GBLOD_POINTS_BLOCK16 selects with the quantised node table and draws
 *   the decoded codes (the image then equals the oracle's render of the decoded points);
 *   GBLOD_ERR_INVALID_ARG if the octree does not hold the chosen form. */
gblod_status gblod_render(gblod_renderer *r, const gblod_octree *octree, const gblod_camera *camera,
                          const gblod_render_params *params, uint8_t *d_image, uint64_t *d_accum, void *stream);

/* Fitting a node's stored points (abstract: an LOD image "indistinguishable from a full
 * rendering"; octree paragraph: a node's n points stand for all of its particles).
 *
 * gblod_octree_node_points copies node `node`'s stored points (its n_max representatives, or a
 * leaf's particles) to d_pts4 (count x 4 float: x, y, z, weight) and d_hs (count float), device to
 * device, on `stream`; either may be NULL to ask for *count (= the node's point_count) only.
 * gblod_octree_node_members copies the input indices (or ids) of the node's member particles, in
 * (key, id) order, to d_ids (count uint32; NULL: *count only).
 * gblod_octree_set_points overwrites the node's stored points with `count` new ones (count must
 * equal its point_count; d_pts4 count x 4 float, d_hs count float, device pointers).  The node's
 * particle bounds (bmin, bmax) and h_cull, and those of every ancestor, grow to cover the new
 * points (a coordinate or h enters the bounds as v + 0, so -0 counts as +0), so culling stays
 * conservative; the written points' pt_src entries become 0xFFFFFFFF (they copy no particle);
 * w_rep keeps the subselection's weight while each written point carries its own weight; 16-bit
 * block codes, if present, are dropped (run gblod_octree_quantize again).  All three wait for
 * `stream`.  GBLOD_ERR_INVALID_ARG for a node index out of range, a wrong count, or an octree
 * without fp32 points. */
gblod_status gblod_octree_node_points(const gblod_octree *octree, uint32_t node, float *d_pts4, float *d_hs,
                                      uint32_t *count, void *stream);
gblod_status gblod_octree_node_members(const gblod_octree *octree, uint32_t node, uint32_t *d_ids,
                                       uint32_t *count, void *stream);
gblod_status gblod_octree_set_points(gblod_octree *octree, uint32_t node, const float *d_pts4, const float *d_hs,
                                     uint32_t count, void *stream);

/* One part of a split frame (multi-GPU sharding of one LOD frame, replica octrees on every GPU).
 * The frame's node selection (depth paragraph) is computed in full; of the nodes it emits, part
 * `part` of `n_parts` keeps those whose index in the octree's node table is congruent to `part`
 * modulo `n_parts` (the same on every replica, since the node table is deterministic), and draws
 * only their points into d_accum (height x width uint64, overwritten).  The parts' images sum, as
 * integers, to exactly the frame gblod_render draws: every emitted node belongs to one part and the
 * accumulation is an exact integer sum.  Sum the parts (one int64 sum-reduce, e.g. NCCL), then call
 * gblod_tonemap once.  GBLOD_ERR_INVALID_ARG unless 0 <= part < n_parts and d_accum is given. */
gblod_status gblod_render_part(gblod_renderer *r, const gblod_octree *octree, const gblod_camera *camera,
                               const gblod_render_params *params, int32_t part, int32_t n_parts, uint64_t *d_accum,
                               void *stream);

/* R4 alone: the log tone map of a caller's accumulation image d_accum (height x width uint64, e.g.
 * the summed parts of a split frame) into d_image (height x width uint8), with the tone-map fields
 * of `params` (automatic or fixed range), exactly as gblod_render maps its own accumulation. */
gblod_status gblod_tonemap(gblod_renderer *r, const uint64_t *d_accum, int32_t width, int32_t height,
                           const gblod_render_params *params, uint8_t *d_image, void *stream);

/* Brute-force frame: R2-R4 over every particle (d_xyz n x 3, d_mass n, d_h n), no tree
 * (params->point_format is ignored: the fp32 particles are drawn). */
gblod_status gblod_render_bruteforce(gblod_renderer *r, const float *d_xyz, const float *d_mass, const float *d_h,
                                     uint64_t n, const gblod_camera *camera, const gblod_render_params *params,
                                     uint8_t *d_image, uint64_t *d_accum, void *stream);

typedef struct {
    uint64_t nodes_selected; /* R1 output */
    uint64_t points;         /* points fed to R2 */
    uint64_t splats;         /* points drawn after culling */
    uint64_t pairs;          /* (tile, splat) records; a point whose clipped pixel box is at most
                                8 x 8 pixels is drawn without records (added to the image directly) */
    uint64_t tiles;
    uint64_t amplitude_lo, amplitude_hi; /* sum of drawn amplitudes */
    uint64_t pixel_updates;  /* (splat, pixel) pairs inside the kernel support (0 unless the frame
                                was rendered with GBLOD_RENDER_COUNT_UPDATES) */
    uint64_t pixel_updates_total; /* the same, summed over every frame of this renderer */
} gblod_frame_stats;

/* Waits for `stream`, then reports the sticky device status (GBLOD_OK or GBLOD_ERR_RANGE /
 * GBLOD_ERR_DEVICE_TIMEOUT) and, if reset != 0, clears it. */
gblod_status gblod_renderer_status(gblod_renderer *r, void *stream, int reset);

/* Counters of the last frame; waits for `stream`. */
gblod_status gblod_renderer_stats(gblod_renderer *r, void *stream, gblod_frame_stats *out);

/* Node indices selected by the last LOD frame (any order), up to `cap`; *count gets the total.
 * Waits for `stream`. */
gblod_status gblod_renderer_last_selection(gblod_renderer *r, void *stream, uint32_t *h_nodes, uint64_t cap,
                                           uint64_t *count);

/* ----------------------------------------------------------------- batched views */
/* Many views in one set of launches (the paper's interactive use renders a stream of views; a
 * serving system renders many viewers' views at once).  Each view has its own camera, resolution
 * and octree (e.g. one octree per timestep).  Every view's images equal what gblod_render gives for
 * it alone, bit for bit. */
typedef struct {
    const gblod_octree *octree; /* the view's octree */
    gblod_camera camera;
    uint8_t *d_image;           /* height x width uint8, or NULL */
    uint64_t *d_accum;          /* height x width uint64 fixed-point image; required */
} gblod_view;

/* Sizes the renderer's batch scratch for batches no larger than `views` (node counts, tiles,
 * pixels) with room for `record_capacity` (tile, splat) records (0 = 2^28, at most 2^32 - 1).
 * A batch holds 1..65535 views.
 * Allocates; waits for `stream`. */
gblod_status gblod_renderer_reserve_batch(gblod_renderer *r, const gblod_view *views, int32_t n_views,
                                          const gblod_render_params *params, uint64_t record_capacity,
                                          void *stream);

/* Renders every view (R1-R4).  Enqueues work on `stream` and returns without waiting: no host
 * synchronisation and no allocation happen inside, so the call can be recorded into a CUDA graph.
 * Requires a prior gblod_renderer_reserve_batch covering this batch (GBLOD_ERR_INVALID_ARG
 * otherwise).  A batch whose (tile, splat) records exceed the reserved capacity sets the sticky
 * capacity status (gblod_renderer_status returns GBLOD_ERR_CAPACITY) and its images are invalid.
 * The per-view constants are passed by value to a kernel at enqueue time, so the caller's arrays
 * may be reused as soon as the call returns. */
gblod_status gblod_render_batch(gblod_renderer *r, const gblod_view *views, int32_t n_views,
                                const gblod_render_params *params, void *stream);

/* Autotuner: renders the batch with each candidate screen tile (16x16, 32x16, 16x32, 32x32, 64x16)
 * and keeps the fastest in params_inout->tile_w/tile_h (the image is the same for every tile);
 * *best_ms gets its time.  Candidates whose records overflow `record_capacity` are not eligible
 * (GBLOD_ERR_CAPACITY if none fits).  Reserves as needed and waits for `stream`.  The winner is
 * cached per (device, multiset of view resolutions, kernel, point format, record capacity,
 * power-of-two class of the batch's drawn splats, measured by one render with the caller's tile);
 * a later call with the same key renders once and returns the cached tile and time. */
gblod_status gblod_autotune_tiles(gblod_renderer *r, const gblod_view *views, int32_t n_views,
                                  gblod_render_params *params_inout, uint64_t record_capacity, void *stream,
                                  double *best_ms);

/* Forgets every cached autotuner result (process-wide). */
void gblod_autotune_cache_clear(void);

/* ----------------------------------------------------------------- differentiation */
/* Float splat of n points (d_xyz n x 3, weights d_w n, log smoothing lengths d_logh n) into
 * n_views images of one resolution (d_images n_views x height x width float32, overwritten).
 * Reading for fitting representatives to the full-data image (abstract: the LOD image should be
 * indistinguishable from a full rendering): sigma = clamp(f exp(l)/z_c, sigma_min, sigma_max),
 * kernel (exp(-r^2/2 sigma^2) - e^-4.5) / (2 pi sigma^2 (1 - 5.5 e^-4.5)) for r < 3 sigma,
 * fp32 accumulation (sum order not fixed: results agree to rounding, not bit for bit).  Waits for
 * `stream` once per chunk of views to size its scratch. */
gblod_status gblod_diff_render(gblod_renderer *r, const float *d_xyz, const float *d_w, const float *d_logh,
                               uint64_t n, const gblod_camera *cams, int32_t n_views,
                               const gblod_render_params *params, float *d_images, void *stream);

/* Adjoint of gblod_diff_render: given dL/dI (d_grad_images, same layout as d_images), writes
 * dL/dxyz (n x 3), dL/dw (n) and dL/dlog h (n) (overwritten; zero through a sigma clamp).  Every
 * per-pixel term is recomputed tile by tile; nothing per pixel is stored between the calls. */
gblod_status gblod_diff_backward(gblod_renderer *r, const float *d_xyz, const float *d_w, const float *d_logh,
                                 uint64_t n, const gblod_camera *cams, int32_t n_views,
                                 const gblod_render_params *params, const float *d_grad_images, float *d_grad_xyz,
                                 float *d_grad_w, float *d_grad_logh, void *stream);

/* ----------------------------------------------------------------- fixed-scratch variant */
/* Brute-force frame that allocates no memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- host applications that own the whole
 * device memory budget and hand this library only its input and output buffers, plug-ins whose
 * host forbids device allocation, and real-time loops that must not call cudaMalloc/cudaFree
 * because those calls can block or synchronise the device.
 *
 * Same arguments, results and semantics as gblod_render_bruteforce (identical fixed-point image),
 * except:
 *   - d_accum is required (the caller owns the height x width uint64 output); d_image may be NULL;
 *   - scratch is one statically sized device array inside this library, GBLOD_NOALLOC_SCRATCH_BYTES
 *     bytes, which every GPU that loads the library holds until the process exits;
 *   - the first call on a device also performs that device's set-up (loads the library's device
 *     code and uploads the kernel table); make that first call before any stream capture.  Every
 *     call looks the array's device address up again in the current context (cudaGetSymbolAddress),
 *     so the entry point stays valid across a teardown and re-creation of the device context;
 *   - frames are limited to GBLOD_NOALLOC_MAX_TILES screen tiles (e.g. 4096 x 4096 pixels with
 *     the default 64 x 16 tiles; larger images are rejected with GBLOD_ERR_INVALID_ARG) and to
 *     GBLOD_NOALLOC_MAX_RECORDS (tile, splat) records (a frame that needs more returns
 *     GBLOD_ERR_RANGE before anything is splatted; d_accum is then left unspecified);
 *   - every call shares the one array, so calls that overlap on the GPU (on different streams, or
 *     from different host threads) race and corrupt each other: serialise them;
 *   - the fixed-point range checks are returned directly (GBLOD_ERR_RANGE) since there is no
 *     renderer object to hold a status word; the frame is still completed without the dropped
 *     splats.  The call waits once on `stream` mid-frame, like gblod_render_bruteforce. */
#define GBLOD_NOALLOC_MAX_TILES 16384u /* e.g. 4096 x 4096 pixels with the default 64 x 16 tiles */
#define GBLOD_NOALLOC_MAX_RECORDS 2097152u
#define GBLOD_NOALLOC_SCRATCH_BYTES 34227456u /* 32.6 MiB */
gblod_status gblod_render_bruteforce_noalloc(const float *d_xyz, const float *d_mass, const float *d_h, uint64_t n,
                                             const gblod_camera *camera, const gblod_render_params *params,
                                             uint8_t *d_image, uint64_t *d_accum, void *stream);

/* ----------------------------------------------------------------- stage entry points */
/* A1 alone: 63-bit Morton keys of n points (octree paragraph; q = clamp(floor((x - lo) 2^21 /
 * side)), octant bits (x<<2)|(y<<1)|z, level 1 in bits 62..60). */
gblod_status gblod_morton_keys(const float *d_xyz, uint64_t n, const double root_lo[3], double root_side,
                               uint64_t *d_keys, void *stream);

/* R2 alone, for n points given as float4 (x, y, z, weight) + h: d_out n x 5 int64 =
 * {drawn (1), culled (0) or out of range (-1), U, V, S, Wq}. */
gblod_status gblod_project(const float *d_pts4, const float *d_h, uint64_t n, const gblod_camera *camera,
                           const gblod_render_params *params, int64_t *d_out, void *stream);

/* Returns the memory cached by the library's pool of the current device (see gblod_allocator)
 * to the device, keeping at most keep_bytes; memory still allocated is not touched.  Call it with
 * no library work in flight on the device that is to free memory (freed blocks are released once
 * the work before their cudaFreeAsync has completed).  Errors: GBLOD_ERR_CUDA. */
gblod_status gblod_trim_cache(uint64_t keep_bytes);

/* ----------------------------------------------------------------- instrumentation */
/* Number of kernel launches this library has issued in the process. */
uint64_t gblod_launch_count(void);

/* Kernel ids for the timing probe. */
typedef enum {
    GBLOD_K_ANY = 0,
    GBLOD_K_MORTON, GBLOD_K_SORT_UPSWEEP, GBLOD_K_SORT_SCATTER, GBLOD_K_SCAN, GBLOD_K_BUILD_OTHER,
    GBLOD_K_SEL_HIST, GBLOD_K_SEL_MARK, GBLOD_K_SEL_WRITE, GBLOD_K_SELECT_NODES, GBLOD_K_PROJECT_COUNT,
    GBLOD_K_PROJECT_SCATTER, GBLOD_K_SPLAT, GBLOD_K_TONEMAP, GBLOD_K_RENDER_OTHER,
    GBLOD_K_COUNT_
} gblod_kernel_id;

/* Timing probe: while enabled for `kernel` (GBLOD_K_ANY = none), every launch of that kernel is
 * bracketed by CUDA events on its own stream.  gblod_probe_read waits for the recorded events
 * and returns the summed device time and the number of launches since the probe was enabled. */
gblod_status gblod_probe_enable(int32_t kernel);
gblod_status gblod_probe_read(double *total_ms, uint64_t *launches);

/* Issue-rate probes of the integer instruction mixes the splat kernels execute (the measured
 * ceilings that roofline fractions of the integer-bound kernels are stated against; the paper has
 * no counterpart).  Kinds: ALU = (a ^ b) + c chains (2 ops per step), IMAD = 32-bit multiply-add,
 * IMAD_WIDE = 64-bit accumulation of a 32 x 32 -> 64 product, IMAD_HI = accumulation of the high
 * word of a 32 x 32 product, LDS = conflict-free shared-memory word loads, RADIAL = the radial
 * rule's per-pixel body with every pixel inside the support (unit: pixel updates), SEPARABLE = the
 * separable rule's per-pixel body (unit: pixel updates).  One untimed and one timed launch of
 * (SMs x resident blocks) x 256 threads, `iters` outer iterations per thread (1..2^24), enqueued
 * on `stream` and timed with CUDA events; the call waits for them.  Out: *ms = device time of the
 * timed launch, *units = operations (or pixel updates) it performed.  It allocates (and frees) a
 * small result buffer with cudaMallocAsync. */
typedef enum {
    GBLOD_MB_ALU = 0, GBLOD_MB_IMAD, GBLOD_MB_IMAD_WIDE, GBLOD_MB_IMAD_HI, GBLOD_MB_LDS, GBLOD_MB_RADIAL,
    GBLOD_MB_SEPARABLE, GBLOD_MB_COUNT_
} gblod_microbench_kind;
gblod_status gblod_microbench(int32_t kind, uint32_t iters, void *stream, double *ms, double *units);

const char *gblod_status_string(gblod_status s);
const char *gblod_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GBLOD_H */
