/*
 * lfdepth — superpixel light-field depth estimation on one NVIDIA GB300
 * (sm_103a): the data-parallel hot path of Chuchvara, Barsi, Gotchev,
 * "Fast and Accurate Depth Estimation from Sparse Light Fields"
 * (arXiv 1812.06856), Section III-B (plane sweep), III-C (propagation and
 * plane refinement with the energy of Eq. 3-11) and III-E (all superpixels of
 * all views in parallel, ping-pong plane buffers).
 *
 * Conventions used by every call
 *  - Cameras: a world point X maps to camera coordinates x = R X + t; the
 *    pixel is K x / x_z, pixel centres at integer coordinates (0..W-1,
 *    0..H-1), x right, y down, z forward.  K must be pinhole (last row 0 0 1).
 *  - Colours are RGB in [0,1]: RGBA8 texels are value/255; the alpha channel
 *    is ignored.
 *  - A point projected into view i at (x, y) lies in that view iff it is in
 *    front of both cameras and -1/2 <= x < W - 1/2, -1/2 <= y < H - 1/2 (the
 *    image's texture area: its nearest pixel floor(x + 1/2), floor(y + 1/2)
 *    is a pixel of view i).  Bilinear samples clamp the coordinates to the
 *    outermost pixel centres (clamp to edge).
 *  - Superpixels: label maps are row-major int32 H x W per view with values in
 *    [0, grid_w * grid_h); label = gy * grid_w + gx places the superpixel on a
 *    regular grid whose 8-neighbourhood is the paper's neighbour system
 *    (Section III-A).  Empty labels are allowed.
 *  - Planes: one float4 {d, nx, ny, nz} per superpixel, in the camera frame of
 *    its view: d > 0 is the depth (camera z) at the superpixel centroid and n
 *    the unit normal facing the camera (Section II, III-A: "a single depth value
 *    at a superpixel centroid and a normal vector").  {0,0,0,0} marks an
 *    empty superpixel / no plane.
 *  - Depth maps: float32 H x W per view, camera z of the pixel's superpixel
 *    plane along the pixel ray, 0 where there is none.
 *  - Streams: every call that takes `stream` (a cudaStream_t, NULL = legacy
 *    default stream) only enqueues work on it and returns; inputs must stay
 *    alive and outputs untouched until the stream has passed the call.
 *    Calls documented as synchronous wait for their own work.
 *  - Errors: every call returns an lfd_status and never throws; after a
 *    failure lfd_last_error(ctx) describes it.  Invalid arguments are
 *    reported before anything is enqueued.  Device-side checks (labels out of
 *    range) raise a status word that the next lfd_synchronize() reports as
 *    LFD_ERR_DEVICE_CHECK.
 *  - Ownership: the caller owns every buffer it passes; the context owns its
 *    workspace (superpixel lists and statistics, sampling textures, rasterised
 *    maps, ping-pong planes) and frees it in lfd_destroy().
 *  - One context serves one bound input (one light field, or n of them
 *    through lfd_estimate_batch) at a time and is not thread safe; use one
 *    context per concurrent input.
 */
#ifndef LFDEPTH_H
#define LFDEPTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LFD_VERSION 2
#define LFD_MAX_NEIGHBOR_VIEWS 8   /* |N(v)| of Eq. 2 / Eq. 8 is at most this */
#define LFD_MAX_VIEWS 256
#define LFD_MAX_LABELS 4096
#define LFD_MAX_ITER_INDEX 64      /* iteration index I of Eq. 4 (plus warm offset) */
#define LFD_MAX_DIM 32767          /* image width / height */
/* per-query record of lfd_score(): LFD_TERMS_HEAD scalars then, for each
 * neighbour view k < LFD_MAX_NEIGHBOR_VIEWS, LFD_TERMS_PER_VIEW scalars */
#define LFD_TERMS_HEAD 4           /* E, E_s, E_c, TSSD sum */
#define LFD_TERMS_PER_VIEW 6       /* S_i, V_i, O_i, |Omega_i|, |X_i|, |Y_i| */
#define LFD_TERMS_STRIDE (LFD_TERMS_HEAD + LFD_MAX_NEIGHBOR_VIEWS * LFD_TERMS_PER_VIEW)

typedef int32_t lfd_status;
enum {
    LFD_OK = 0,
    LFD_ERR_INVALID_ARG = 1,   /* a documented precondition does not hold */
    LFD_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    LFD_ERR_OOM = 3,           /* device or pinned memory allocation failed */
    LFD_ERR_BUDGET = 4,        /* the workspace would exceed the context's HBM budget */
    LFD_ERR_TIMEOUT = 5,       /* a bounded wait ran out */
    LFD_ERR_DEVICE_CHECK = 6,  /* a device-side input check failed (see lfd_last_error) */
    LFD_ERR_BUSY = 7,           /* a queue bound was reached (lfd_server_submit) */
    LFD_ERR_STATE = 8          /* call order: e.g. lfd_iterate before lfd_set_input */
};

typedef enum {
    LFD_RGBA8 = 0,      /* 4 x uint8 per texel */
    LFD_RGBA_F16 = 1,   /* 4 x IEEE half per texel */
    LFD_RGBA_BF16 = 2,  /* 4 x bfloat16 per texel */
    LFD_RGBA_F32 = 3    /* 4 x float per texel */
} lfd_pixfmt;

typedef struct {
    double K[9];        /* row-major intrinsics, last row 0 0 1 */
    double R[9];        /* row-major world -> camera rotation */
    double t[3];        /* world -> camera translation */
    int32_t width, height;
} lfd_camera;

typedef struct {
    int32_t num_views;                   /* V >= 2 */
    int32_t fmt;                         /* lfd_pixfmt of every view */
    const lfd_camera *cams;              /* host array [V] */
    const void *const *views;            /* host array [V] of image pointers (device memory, or host
                                            memory for lfd_estimate_host), H rows of pitch bytes */
    const int64_t *view_pitch_bytes;     /* host array [V]; NULL or 0 entries = width * texel size */
    const int32_t *const *labels;        /* host array [V] of label-map pointers, tightly packed H x W */
    const int32_t *grid_w;               /* host array [V] */
    const int32_t *grid_h;               /* host array [V] */
} lfd_lightfield;

/* Parameters.  lfd_params_default() fills the values in brackets. */
typedef struct {
    double d_min, d_max;         /* scene depth range, 0 < d_min < d_max (Section III-B) */
    int32_t num_labels;          /* L inverse-depth levels of the sweep [64], 1..LFD_MAX_LABELS */
    int32_t iterations;          /* refinement iterations [5] (Section IV-A) */
    double T;                    /* truncation of Eq. 1 on RGB in [0,1] [0.04] */
    double sigma;                /* Eq. 6 / Eq. 10 Gaussian width; 0 = 2 x bin width of the domain [0] */
    double alpha;                /* Eq. 7 colour width [0.1] */
    double eta;                  /* Eq. 11 occlusion regulariser [0.5] */
    int32_t kernel_size_init;    /* initial kernel size in pixels, 0 = smallest image dimension
                                    (Section IV-A) [0] */
    double kernel_step_sp;       /* kernel step in superpixels (Section IV-A) [5] */
    int32_t max_neighbor_views;  /* |N(v)|: nearest camera centres, 1..8, 0 = 8 [0] */
    int32_t depth_domain;        /* Gaussians of Eq. 6/10 and the X/Y split: 0 inverse depth, 1 depth [0] */
    int32_t jitter;              /* 1: one uniform sample per inverse-depth bin (Section III-B);
                                    0: bin centres [1] */
    uint32_t term_mask;          /* bit0 smoothness E_s, bit1 consistency E_c, bit2 occlusion O [7] */
    int32_t sweep_frame;         /* sweep planes fronto-parallel to 0 the view's camera, 1 the world [0] */
    uint64_t seed;               /* jitter seed [0x5EED] */
    int32_t lf_index;            /* light-field index mixed into the jitter key [0] */
    double xy_eps;               /* relative tolerance of the X/Y split of Eq. 10/11 [0] */
    int32_t warm_iter_offset;    /* iteration I of Eq. 4 is iter + offset (warm starts) [0] */
    /* Flagged variant, not in the paper (which never refines depth continuously):
     * after the 8 triangle normals, the refinement step also scores
     * perturb_samples random planes around the propagated plane (d, n): depth
     * d (1 + r (2u - 1)), normal normalize(n + r (2u' - 1, 2u'' - 1, 2u''' - 1)),
     * r = perturb_scale 2^(1 - I), u from SplitMix64 of seed ^ 0x5045525455524231
     * and key ((((lf*2^12 + v)*2^20 + s)*2^7 + I)*2^7 + 4k + j); the first
     * strictly better one wins.  0..24 samples [0 = off], scale >= 0 [0.05]. */
    int32_t perturb_samples;
    double perturb_scale;
} lfd_params;

/* one hypothesis for lfd_score(): plane {d, n} of superpixel `sp` of `view` */
typedef struct {
    int32_t view, sp;
    float d, nx, ny, nz;
} lfd_query;

typedef struct lfd_ctx lfd_ctx;

/* ---- library ---------------------------------------------------------- */

int32_t lfd_version(void);
/* ABI check for bindings: writes sizeof(lfd_camera), sizeof(lfd_lightfield),
 * sizeof(lfd_params), sizeof(lfd_query), sizeof(lfd_batch_options),
 * sizeof(lfd_result) into out[0..5]. */
void lfd_struct_sizes(int32_t *out);
const char *lfd_status_string(lfd_status s);
void lfd_params_default(lfd_params *p);

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * workspace the context may allocate (0 = no bound).  *out receives the
 * context; allocation is deferred to lfd_set_input. */
lfd_status lfd_create(lfd_ctx **out, int32_t device, uint64_t hbm_budget_bytes);
/* Free the context and its workspace (waits for its work first). */
lfd_status lfd_destroy(lfd_ctx *ctx);
/* Message of the last failure on ctx (never NULL; "" after success). */
const char *lfd_last_error(const lfd_ctx *ctx);

/* ---- staged hot path -------------------------------------------------- */

/* Bind a light field and parameters to the context: validate them, size the
 * workspace (LFD_ERR_BUDGET past the budget), copy the cameras, choose each
 * view's neighbour views N(v) (the min(V-1, max_neighbor_views) nearest camera
 * centres, nearer first, ties to the lower index), build each view's sampling
 * texture from `views`, and build the superpixels (Section III-A; step a1):
 * per label the row-major pixel list, the centroid, the mean colour C_Omega
 * and the minimum colour similarity to the present 8-neighbours (Eq. 11).
 * Views and labels are device pointers and are read only during this call's
 * stream work.  Asynchronous. */
lfd_status lfd_set_input(lfd_ctx *ctx, const lfd_lightfield *lf, const lfd_params *p, void *stream);

/* Number of superpixels (grid_w * grid_h) of `view` of the bound light field. */
lfd_status lfd_num_superpixels(const lfd_ctx *ctx, int32_t view, int32_t *out);

/* Plane sweep (Section III-B, Eq. 1-2; steps a2-a4): for every superpixel of
 * every view, L fronto-parallel planes at inverse depths
 * 1/d_max + (k + u_k) (1/d_min - 1/d_max) / L, u_k uniform in [0,1) per
 * superpixel and label (SplitMix64 of seed ^ key, key = ((lf*2^12 + v)*2^20 +
 * s)*2^12 + k), are scored by the sum over N(v) and the superpixel's pixels
 * of min(T, SSD) with bilinear sampling through the plane-induced homography
 * (a projection outside view i or behind a camera costs T); the lowest cost
 * wins (lowest k on ties).
 *   planes_out: host array [V] of device float4[S_v] (required).
 *   label_out:  host array [V] of device int32[S_v] winning k, -1 if empty (nullable).
 *   cost_out:   host array [V] of device float[S_v * L], all costs (nullable).
 * Asynchronous. */
lfd_status lfd_plane_sweep(lfd_ctx *ctx, float *const *planes_out, int32_t *const *label_out,
                           float *const *cost_out, void *stream);

/* Depth rasteriser (step a5): every pixel's depth from its superpixel's plane
 * (the plane's camera z along the pixel ray; 0 if the plane is behind the
 * camera or missing), into the context's sampling maps used by lfd_iterate's
 * visibility test of Eq. 10, and into depth_out if given.
 *   planes: host array [V] of device float4[S_v].
 *   depth_out: host array [V] of device float[H*W] (nullable).
 * Asynchronous. */
lfd_status lfd_rasterize(lfd_ctx *ctx, const float *const *planes, float *const *depth_out, void *stream);

/* One refinement iteration (Section III-C, III-E; steps a5-a7): rasterise
 * planes_in, then for every superpixel of every view, in parallel and reading
 * only planes_in (Jacobi): propagation — the current plane and the planes of
 * the kernel's superpixels (the 8 neighbours, then along 8 compass rays the
 * cells at r_k = max(1, floor(k Size_I/Steps_I + 0.5)), k = 1..Steps_I, with
 * Size_I = Size_init/I, Steps_I = max(1, floor(Steps_init/I)) (Eq. 4)), each
 * re-anchored at the own centroid and rejected if its depth there leaves
 * [d_min, d_max] or it is grazing (|n . ray| < 0.1), replace the current plane
 * when E = E_c E_s (Eq. 3) is strictly greater; refinement — the normals of the
 * 8 ring triangles (own centroid at the new depth and two consecutive
 * neighbour centroids at their depths; Fig. 3b) replace the normal on strict
 * improvement.  iter is the 1-based I of Eq. 4 (warm_iter_offset is added).
 *   planes_in / planes_out: host arrays [V] of device float4[S_v]; must not alias.
 *   choice_out: host array [V] of device int32[2*S_v]: propagation candidate index
 *               (0 = current), refinement triangle (-1 = none) (nullable).
 *   energy_out: host array [V] of device float[2*S_v]: E after propagation and after
 *               refinement (nullable).
 * Asynchronous. */
lfd_status lfd_iterate(lfd_ctx *ctx, int32_t iter, const float *const *planes_in, float *const *planes_out,
                       int32_t *const *choice_out, float *const *energy_out, void *stream);

/* Whole frame (steps a1-a8): lfd_set_input, then the plane sweep (or
 * warm_planes when given), then p->iterations iterations ping-ponging two
 * workspace buffers, then the final planes into planes_out and their depth
 * maps into depth_out (nullable).  All pointers in lf and the outputs are
 * device pointers; warm_planes is a host array [V] of device float4[S_v] or
 * NULL.  Asynchronous. */
lfd_status lfd_estimate(lfd_ctx *ctx, const lfd_lightfield *lf, const lfd_params *p,
                        const float *const *warm_planes, float *const *planes_out, float *const *depth_out,
                        void *stream);

/* lfd_estimate with every image, label map and output in HOST memory: the
 * call copies the inputs to the device, runs the frame and copies the planes
 * and depth maps back.  Pinned host memory makes the copies asynchronous;
 * the call returns after enqueueing and the results are valid once the
 * stream has passed it (lfd_synchronize). */
lfd_status lfd_estimate_host(lfd_ctx *ctx, const lfd_lightfield *lf_host, const lfd_params *p,
                             float *const *planes_out_host, float *const *depth_out_host, void *stream);

/* ---- SLIC superpixels (step before the hot path) ----------------------- */

/* SLIC segmentation (Achanta et al. 2012; the paper segments every view with
 * a GPU SLIC before Section III-A) into label maps the rest of the path takes
 * as they are: label = cy * grid_w + cx of the winning seed cell.
 * CIELAB (sRGB companding, D65); one seed per cell of the grid whose
 * boundaries are at round(k W / grid_w) (half up), at the cell centre with the
 * colour of its nearest pixel; each iteration assigns every pixel to the
 * nearest of the 3x3 seed cells around its own cell by
 * D^2 = |dLab|^2 + (compactness / S)^2 |dxy|^2, S = sqrt(W H / (grid_w grid_h))
 * (ties to the first cell in row-major order), then moves each centre to the
 * mean of its pixels; a final assignment writes the labels.  No connectivity
 * post-processing.  A pixel whose colour is not finite keeps its own cell and
 * does not enter the means; the means take Lab values clamped to [-256, 256]
 * (every sRGB colour in [0,1] is inside) in fixed point (2^-18). 
 *   views, view_pitch_bytes (nullable = packed), width, height, grid_w,
 *   grid_h: arrays [n] (host); images and labels_out[v] (int32 H*W) on the
 *   device.  centres_in / centres_out (nullable; entries float[grid_w*grid_h*5]
 *   {L, a, b, x, y} on the device): start from given centres instead of the
 *   seeds / receive the centres the final assignment used.
 * Scratch is allocated in the context on first use.  Asynchronous. */
lfd_status lfd_slic(lfd_ctx *ctx, int32_t n, const void *const *views, const int64_t *view_pitch_bytes, int32_t fmt,
                    const int32_t *width, const int32_t *height, const int32_t *grid_w, const int32_t *grid_h,
                    double compactness, int32_t iterations, int32_t *const *labels_out,
                    const float *const *centres_in, float *const *centres_out, void *stream);

/* ---- depth fusion (step after the hot path) ---------------------------- */

/* Stability-based depth fusion (Section III-D) of one depth map per bound
 * view, light field by light field.  Each view in turn is the reference:
 * every pixel of every other view of its light field with a depth > 0 is
 * lifted to a 3-D point and projected to the reference's nearest pixel
 * (floor(x + 0.5), valid iff in front and 0 <= x <= W-1, 0 <= y <= H-1);
 * per other view the point of smallest depth wins a pixel.  Each depth
 * candidate of a reference pixel (its own depth when > 0 and one per other
 * view) gets stability = #candidates with |z - z_c| <= tau z_c minus #others;
 * the closest candidate with stability >= 0 is written (0 if none).
 *   depth_in / depth_out: host arrays [V] of device float[H*W] (the layout of
 *   lfd_estimate's depth maps); must not alias.  tau > 0 (0.01 = 1 %).
 * The z-buffers (V_l - 1 planes per view of the largest light field) are
 * allocated on first use outside the context's budget.  Asynchronous. */
lfd_status lfd_fuse(lfd_ctx *ctx, const float *const *depth_in, float *const *depth_out, double tau, void *stream);

/* ---- batched frames --------------------------------------------------- */

/* Launch options of lfd_estimate_batch (lfd_batch_options_default fills
 * autotune 0, graph 0, sweep_threads 256, sweep_persistent 1, prop_blocks 8,
 * prop_persistent 1, prop_batch 32, order_bands 16, prop_coop 0). */
typedef struct {
    int32_t autotune;          /* 1: the first call with a new argument signature times, on its
                                  own input, the sweep (128/256 threads x grid/persistent x
                                  1/16 row bands in the work order) and the propagation (7/8
                                  CTAs per SM x grid/persistent warps/cooperative CTAs x 16/32
                                  candidates per batch x 1/16 row bands, timed on the first and
                                  the last iteration) and keeps the fastest of each; the shape
                                  fields are then ignored */
    int32_t graph;             /* 1: the frame's device work is captured as a CUDA graph on the
                                  first call; a later call whose signature (every pointer, size,
                                  camera, parameter and option) is identical replays it, reading
                                  the current contents of the same image and label buffers.
                                  Needs a non-default stream. */
    int32_t sweep_threads;     /* 128 or 256 (0 = 256): labels scored in parallel per superpixel */
    int32_t sweep_persistent;  /* 1: persistent sweep CTAs take superpixels from a queue ordered
                                  by size (pixel-slot class ceil(n/32)), largest first */
    int32_t prop_blocks;       /* 7 or 8 (0 = 8) resident propagation CTAs per SM */
    int32_t prop_persistent;   /* 1: persistent propagation warps over the same ordered queue */
    int32_t prop_batch;        /* 16 or 32 (0 = 32): candidate planes a warp scores per pass over the
                                  neighbour views (their footprints share L1 across the pass) */
    int32_t order_bands;       /* 1 or 16 (0 = 16): row bands of the work orders inside a size class
                                  (16: the superpixels in flight cover the same rows of every view) */
    int32_t prop_coop;         /* 1 (with prop_persistent): the 4 warps of a propagation CTA update
                                  one superpixel together, its candidates split between them, so
                                  they gather from one footprint per neighbour view (L1 reuse);
                                  0: one superpixel per warp.  Same results either way; on the
                                  16 x 1080p and 8 x 1024x768 frames 0 is faster (the kernel is
                                  issue-bound and the split costs instructions and barriers). */
} lfd_batch_options;

void lfd_batch_options_default(lfd_batch_options *o);

/* Several light fields (e.g. the frames of several rigs) in ONE pass of the
 * hot path (Section III-E applied across light fields): every superpixel of
 * every view of every light field is one work item of the same sweep and
 * propagation launches.  Each light field keeps its own cameras, neighbour
 * views (within the light field), parameters and jitter key; results are the
 * same as n separate lfd_estimate calls.  Light fields of one call must share
 * the pixel format, depth_domain and sweep_frame; a light field with fewer
 * iterations than the largest passes its planes through the remaining ones.
 *   lfs, params:  arrays [n] (host memory); images and labels are device pointers.
 *   planes_out:   host array [n] of host arrays [V_l] of device float4[S_v] (required).
 *   depth_out:    host array [n] of host arrays [V_l] of device float[H*W] (nullable,
 *                 entries nullable).
 *   options:      NULL = defaults.
 * After the call the context is bound to all n light fields, numbered
 * globally (light field 0's views first) for the staged calls.  Asynchronous,
 * except that autotuning (first call of a signature) synchronises the stream. */
lfd_status lfd_estimate_batch(lfd_ctx *ctx, int32_t n, const lfd_lightfield *lfs, const lfd_params *params,
                              float *const *const *planes_out, float *const *const *depth_out,
                              const lfd_batch_options *options, void *stream);

/* lfd_estimate_batch with warm starts (the frames of rigs whose previous
 * planes are kept, as a frame server does; the paper processes every light
 * field from scratch).  warm_planes: host array [n]; entry l is NULL (light
 * field l starts cold from the plane sweep) or a host array [V_l] of device
 * float4[S_v] planes it starts from instead: it takes no part in the sweep
 * and runs params[l].iterations iterations with params[l].warm_iter_offset
 * added to I (Eq. 4).  warm_planes itself may be NULL (all cold; the same
 * as lfd_estimate_batch).  Warm planes are read before planes_out is
 * written, so warm_planes[l][v] may equal planes_out[l][v].  Results equal n
 * separate lfd_estimate calls with the same warm planes.  options->graph
 * must be 0 when any light field is warm.  Asynchronous. */
lfd_status lfd_estimate_batch_warm(lfd_ctx *ctx, int32_t n, const lfd_lightfield *lfs, const lfd_params *params,
                                   const float *const *const *warm_planes, float *const *const *planes_out,
                                   float *const *const *depth_out, const lfd_batch_options *options, void *stream);

/* Device workspace (bytes) that binding these n light fields allocates: the
 * figure lfd_create's hbm_budget_bytes is checked against.  Reads only the
 * cameras, grid sizes and pixel format. */
lfd_status lfd_workspace_required(int32_t n, const lfd_lightfield *lfs, uint64_t *bytes);

/* The launch shape in use: out[0..6] = sweep_threads, sweep_persistent,
 * prop_blocks, prop_persistent, prop_batch, order_bands, prop_coop. */
lfd_status lfd_launch_config(const lfd_ctx *ctx, int32_t *out);

/* Homography specialisations of the plane-induced homography A(g) = P + q g^T
 * (Section III-B; the pair's P = K_i R_rel K_v^-1, q = K_i t_rel).  When
 * binding an input the library classifies all its (view, neighbour view)
 * pairs together:
 *   0 general:     any cameras;
 *   1 affine:      every pair has P row 3 = (0, 0, P22) and q_z = 0 (parallel
 *                  optical axes, camera centres at equal depth): the
 *                  homogeneous coordinate of a sample is the same for all
 *                  pixels of a hypothesis, one reciprocal per (hypothesis,
 *                  view); results are the general form's, value for value;
 *   2 translation: affine and P's upper 2 x 2 block = P22 I to 1e-12
 *                  (rectified cameras with equal intrinsics): a
 *                  fronto-parallel sweep plane moves every pixel by one
 *                  vector, whose integer part and fraction the sweep takes in
 *                  FP64; its costs differ from the general form's by the
 *                  rounding of the sample position only (the general form
 *                  rounds absolute positions to FP32; the propagation uses
 *                  form 1).
 * lfd_set_pair_forms(ctx, max_form): the largest form the context may use
 * for inputs bound after the call (0, 1 or 2; default 2; LFD_ERR_INVALID_ARG
 * otherwise); drops a captured CUDA graph.
 * lfd_pair_form(ctx, &form): the form of the bound input (LFD_ERR_STATE
 * before one is bound). */
lfd_status lfd_set_pair_forms(lfd_ctx *ctx, int32_t max_form);
lfd_status lfd_pair_form(const lfd_ctx *ctx, int32_t *form);

/* ---- serving ---------------------------------------------------------- */

/* A frame server: several rigs (camera arrays, each a stream of light-field
 * frames) share one GPU by continuous batching.  Submitted frames wait in one
 * queue in arrival order.  A dispatcher thread owned by the server watches
 * `max_slots` slots (a context and a CUDA stream each); whenever a slot is
 * free it takes every queued frame that can run now -- at most one frame per
 * rig, from rigs with no frame on the device, all warm or all cold, as many
 * as the HBM budget allows -- and runs them as one lfd_estimate_batch_warm
 * call on that slot's stream.  Frames that arrive while batches run join the
 * next batch a freed slot forms; frames of one rig run in submission order.
 * Each frame's result is the same whether it ran alone or in a batch.
 *
 * Warm start (not in the paper, where every frame is independent): the first
 * frame of a rig (or the first after its layout changes) runs the plane sweep
 * and params->iterations iterations; every later frame starts from the rig's
 * previous planes and runs warm_iterations iterations with
 * warm_iter_offset added to the iteration index of Eq. 4 (defaults 3 and 3:
 * the small kernels of I = 4..6).  warm_iterations = 0 makes every frame cold.
 *
 * Admission: a frame is accepted when its own workspace
 * (lfd_workspace_required) plus every rig's plane state fits
 * hbm_budget_bytes (0 = no bound), else the submit fails with LFD_ERR_BUDGET.
 * A batch is formed only while the workspace it needs, the workspaces the
 * other slots hold (each keeps the largest it has used) and the plane states
 * fit the budget; frames that do not fit wait for a later batch (a frame that
 * fits no slot while every slot is idle completes with LFD_ERR_BUDGET).  At
 * most max_pending_per_rig frames of a rig may be submitted and not yet
 * polled; a submit beyond that returns LFD_ERR_BUSY (the caller drops or
 * retries the frame).  Server calls may come from one caller thread at a
 * time. */
typedef struct lfd_server lfd_server;

typedef struct {
    uint64_t req_id;
    int32_t rig_id;
    int32_t warm;              /* 1: started from the rig's previous planes */
    int64_t frame;             /* 0-based frame count of the rig */
    int64_t submit_ns;         /* lfd_server_now_ns() at submission */
    int64_t done_ns;           /* lfd_server_now_ns() when the stream reached the end of its batch */
    lfd_status status;
    int32_t slot;              /* slot whose stream ran the frame */
    int64_t start_ns;          /* lfd_server_now_ns() when its batch was launched */
    int32_t batch;             /* frames in that batch */
    int32_t reserved;
} lfd_result;

lfd_status lfd_server_create(lfd_server **out, int32_t device, uint64_t hbm_budget_bytes, int32_t max_slots);
lfd_status lfd_server_destroy(lfd_server *srv);            /* waits for all frames */
const char *lfd_server_last_error(const lfd_server *srv);
/* Warm-start schedule and queue bound (defaults 3, 3, 2). */
lfd_status lfd_server_configure(lfd_server *srv, int32_t warm_iterations, int32_t warm_iter_offset,
                                int32_t max_pending_per_rig);
/* Largest number of frames in one batch (0 = no limit, the default; 1 runs
 * every frame on its own). */
lfd_status lfd_server_set_max_batch(lfd_server *srv, int32_t max_frames);
/* Batches launched and frames they held since the server was created. */
lfd_status lfd_server_stats(lfd_server *srv, int64_t *batches, int64_t *frames);
/* Monotonic clock of the result timestamps, in ns. */
int64_t lfd_server_now_ns(void);

/* Queue one frame of rig `rig_id` (>= 0).  lf and params as for lfd_estimate
 * (device images and labels, which must stay unchanged until the frame is
 * done); planes_out / depth_out are host arrays [V] of device buffers or NULL.
 * The rig's plane state is kept by the server.  Returns at once with
 * *req_id. */
lfd_status lfd_server_submit(lfd_server *srv, int32_t rig_id, const lfd_lightfield *lf, const lfd_params *params,
                             float *const *planes_out, float *const *depth_out, uint64_t *req_id);
/* Wait up to timeout_us (0 = just test, < 0 = no limit) for request req_id.
 * LFD_OK fills *out and forgets the request; LFD_ERR_TIMEOUT if it is still
 * running; LFD_ERR_INVALID_ARG for an unknown id. */
lfd_status lfd_server_poll(lfd_server *srv, uint64_t req_id, int32_t timeout_us, lfd_result *out);
/* The plane state of rig `rig_id` (all views' superpixels in order, float4
 * each) to host memory once its queued frames have run (synchronous; waits
 * up to a minute, then LFD_ERR_TIMEOUT); *n_sp gets the superpixel count;
 * planes_host may be NULL to query it. */
lfd_status lfd_server_export_state(lfd_server *srv, int32_t rig_id, float *planes_host, int64_t cap_sp,
                                   int64_t *n_sp);
/* Replace rig `rig_id`'s plane state (e.g. exported from another server);
 * its next frame starts warm from it.  The rig must have submitted a frame
 * (its layout is known) and n_sp must match. */
lfd_status lfd_server_import_state(lfd_server *srv, int32_t rig_id, const float *planes_host, int64_t n_sp);

/* Wait for the stream and report device-side check failures
 * (LFD_ERR_DEVICE_CHECK) raised by this context's kernels; clears them. */
lfd_status lfd_synchronize(lfd_ctx *ctx, void *stream);

/* Hypotheses scored and pixel-view samples taken by this context's kernels
 * since the last lfd_set_input / lfd_estimate (synchronous). */
lfd_status lfd_counters(lfd_ctx *ctx, uint64_t *hypotheses, uint64_t *samples, void *stream);

/* ---- tracing ------------------------------------------------------------ */

/* Stages timed by the tracer. */
enum {
    LFD_STAGE_SUPERPIXELS = 0,  /* step a1 kernels of lfd_set_input */
    LFD_STAGE_SWEEP = 1,        /* steps a2-a4 */
    LFD_STAGE_RASTER = 2,       /* step a5 (plane coefficients + rasteriser) */
    LFD_STAGE_PROPAGATE = 3,    /* steps a6-a7 */
    LFD_STAGE_FUSION = 4,       /* lfd_fuse (Section III-D) */
    LFD_STAGES = 5
};

/* Enable (1) or disable (0) CUDA-event timing of every kernel launch of the
 * context, recorded on the launching stream around each launch.  Launch
 * counts are kept whether or not timing is enabled. */
lfd_status lfd_profile_enable(lfd_ctx *ctx, int32_t enable);
/* Synchronous: wait for the recorded events, then write per stage the summed
 * kernel time in milliseconds (ms_out[LFD_STAGES], nullable) and the number
 * of launches (launches_out[LFD_STAGES], nullable) since the last read, and
 * reset both. */
lfd_status lfd_profile_read(lfd_ctx *ctx, double *ms_out, int64_t *launches_out);

/* ---- inspection (tests, tools; synchronous) ---------------------------- */

/* Per-hypothesis terms (Eq. 1-11) of nq planes under the state
 * `state_planes` (host array [V] of device float4[S_v], rasterised first):
 * out (host, nq * LFD_TERMS_STRIDE floats) receives per query
 * E, E_s, E_c, the TSSD sum of Eq. 2, then for each neighbour view k:
 * S_k (Eq. 9), V_k (Eq. 10), O_k (Eq. 11), |Omega_k|, |X_k|, |Y_k|.
 * queries: host array [nq]. */
lfd_status lfd_score(lfd_ctx *ctx, const float *const *state_planes, int32_t nq, const lfd_query *queries,
                     float *out, void *stream);

/* Superpixel lists and statistics of `view` (host outputs, any may be NULL):
 * offsets int32[S+1], pixels int32[H*W] (row-major linear index, row-major
 * order inside each superpixel), stats float[S*8] = {cx, cy, r, g, b, minw,
 * count, 0}; neighbours int32[LFD_MAX_NEIGHBOR_VIEWS] of N(view) (-1 padded). */
lfd_status lfd_get_superpixels(lfd_ctx *ctx, int32_t view, int32_t *offsets, int32_t *pixels, float *stats,
                               int32_t *neighbours, void *stream);

/* ---- allocation-free variant -------------------------------------------- */

/* The paper has no counterpart to this entry point: it serves callers that
 * cannot allocate device memory where they need superpixel statistics, e.g.
 * code recorded into a CUDA graph by stream capture (allocation calls are not
 * allowed during capture), real-time loops with a fixed memory plan that may
 * not touch the allocator once running, or hosts whose device allocator
 * belongs to another framework.
 *
 * It computes, for one view, what lfd_set_input computes per superpixel and
 * lfd_get_superpixels reports as stats: stats_out[s*8 + 0..7] = {cx, cy, r, g,
 * b, minw, count, 0} for every label s < grid_w*grid_h (device float array of
 * grid_w*grid_h*8, caller-owned).  labels: device int32 width x height,
 * row-major; image: device texels of `fmt` with pitch_bytes per row (0 = tight);
 * alpha: colour width used for minw (the same value as lfd_params.alpha).
 * Labels outside [0, grid_w*grid_h) are ignored (the regular path rejects
 * them).  An empty label reports what lfd_get_superpixels reports for it:
 * centroid and colour 0, count 0, and as minw the smallest similarity of
 * colour 0 to its non-empty neighbours (1 if none).  Asynchronous on
 * `stream`; allocates nothing.  LFD_ERR_CUDA only when one of this call's
 * launches fails; an error pending on the calling thread from earlier work
 * is left as it is.
 *
 * Its scratch (per-label counts and bounding boxes) is a fixed device array of
 * LFD_NOALLOC_MAX_LABELS entries (1.25 MiB) that every GPU which loads the
 * library holds until exit.  More labels than that: LFD_ERR_INVALID_ARG.  All
 * calls on a device share the array and each call clears the part it uses,
 * so calls whose GPU work overlaps (other streams, unordered host threads)
 * race and must be serialised.  The first call on each device looks up the
 * array's device address with that device current: make it before any stream
 * capture. */
#define LFD_NOALLOC_MAX_LABELS 65536
lfd_status lfd_superpixel_stats_noalloc(const int32_t *labels, const void *image, int32_t width, int32_t height,
                                        int64_t pitch_bytes, int32_t fmt, int32_t grid_w, int32_t grid_h,
                                        double alpha, float *stats_out, void *stream);

/* ---- host logic (no GPU needed) ---------------------------------------- */

/* N(v) for every view: out[v * LFD_MAX_NEIGHBOR_VIEWS + k], -1 padded;
 * *k_out = min(V-1, max_k or 8). */
lfd_status lfd_neighbor_views(const lfd_camera *cams, int32_t V, int32_t max_k, int32_t *out, int32_t *k_out);

/* Kernel offsets of iteration I (Eq. 4, Fig. 3a): (0,0), the 8 neighbours
 * E NE N NW W SW S SE, then ray cells by k (see lfd_iterate) without repeats,
 * as dx,dy pairs into dxdy[2*cap]; returns the count (writes nothing when it
 * exceeds cap).  size_init / steps_init in superpixel cells. */
int32_t lfd_kernel_offsets(int32_t size_init, int32_t steps_init, int32_t I, int32_t *dxdy, int32_t cap);

#ifdef __cplusplus
}
#endif
#endif /* LFDEPTH_H */
