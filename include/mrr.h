/*
 * mrr.h -- C ABI of libmrr, a CUDA (sm_103a) implementation of the multi-resolution
 * rendering method of Besenthal, Maisch and Ropinski, "Multi-Resolution Rendering for
 * Computationally Expensive Lighting Effects" (arXiv 1906.04576).
 *
 * The method (Sec. 3) has three steps, and the entry points follow them:
 *   1. masks   (Sec. 3.1, Sec. 4.1): mrr_edges, mrr_masks
 *   2. render the sub-images at their resolutions where their masks allow
 *              (Sec. 3.2, Sec. 4.1): mrr_shade_level, optionally mrr_blur_level
 *   3. blend   (Sec. 3.3, Sec. 4.2, Eq. (1)): mrr_upsample_merge
 * mrr_render runs all three for one frame; mrr_render_full is the naive
 * full-resolution rendering the paper compares against (Sec. 5).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev, and every pointer inside mrr_gbuffer / mrr_levels, are CUDA
 *    device pointers owned by the caller; the library never frees them.  Host pointers
 *    are named *_host or documented as host.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls only enqueue work on it and return; nothing synchronises except mrr_wait
 *    and mrr_render_host.
 *  - Arguments are validated before anything is launched: a bad argument returns
 *    MRR_EINVAL and launches nothing.  A CUDA failure returns MRR_ECUDA.  The text of
 *    the last failure is available from mrr_last_error(ctx).  No C++ exception
 *    crosses this ABI.
 *  - Level i (0 = full resolution) has scale 2^-i; it is the paper's sub-image i+1
 *    (Sec. 4.2: "c_1 is the full resolution image").  W_i = ceil(W / 2^i),
 *    H_i = ceil(H / 2^i).  Level texel q covers the full-resolution block
 *    [2^i q, 2^i (q+1)) and is evaluated at the pixel s_i(q) = min(2^i q + o_i, W-1),
 *    o_0 = 0, o_i = 2^(i-1).
 *  - Images are row-major, row 0 at the top, with no padding between rows.
 *  - A context is used by one host thread at a time, except mrr_submit, mrr_poll and
 *    mrr_wait, which are thread-safe.
 */
#ifndef MRR_H
#define MRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRR_MAX_LEVELS 4
#define MRR_MAX_SAMPLES 256     /* hemisphere samples (SSAO, SSGI) */
#define MRR_MAX_TAPS 128        /* PCSS blocker-search and filter taps, each */

typedef enum {
  MRR_OK = 0,
  MRR_EINVAL = 1,        /* invalid argument; nothing was launched */
  MRR_ENOMEM = 2,        /* device or host allocation failed */
  MRR_ECUDA = 3,         /* a CUDA call failed; see mrr_last_error */
  MRR_EBUSY = 4,         /* serving queue full / no free slot */
  MRR_ETIMEDOUT = 5,     /* mrr_wait timed out, or a bounded device-side wait gave up */
  MRR_EUNSUPPORTED = 6   /* valid request this build does not support */
} mrr_status;

/* The three lighting effects of Sec. 2.4 / Sec. 4. */
typedef enum { MRR_SSAO = 0, MRR_SSM = 1, MRR_SSGI = 2 } mrr_effect;

/* Storage precision.  MRR_FP32: normals float4, shadow map float, sub-images float.
 * MRR_FP16: normals half4, shadow map half, sub-images half; depth stays float and all
 * arithmetic stays in float either way.  The SSGI direct-light colour is half4 in both. */
typedef enum { MRR_FP32 = 0, MRR_FP16 = 1 } mrr_precision;

/* Per-context configuration.  Table 1 of the paper gives sigma2 / weight per effect. */
typedef struct mrr_config {
  mrr_effect effect;
  mrr_precision precision;
  int num_levels;                 /* L in 1..MRR_MAX_LEVELS; the coarsest level must be enabled */
  float sigma2[MRR_MAX_LEVELS];   /* Gaussian variance of level i's mask blur, in level texels */
  float weight[MRR_MAX_LEVELS];   /* w_i of Eq. (1) */
  int enabled[MRR_MAX_LEVELS];    /* 0 = level not used (Sec. 4: SSGI skips the 1/2 level) */
  float depth_rel;                /* depth edge: |2nd difference| > depth_rel * depth */
  float normal_cos;               /* normal edge: n_p . n_q < normal_cos */
  int force_level0;               /* 1: every pixel at level 0 (a_0 = 1, S_0 = 1) */
  int samples;                    /* hemisphere samples N (SSAO, SSGI), <= MRR_MAX_SAMPLES */
  float radius;                   /* sampling radius r (view-space units) */
  float ao_bias;                  /* SSAO depth bias */
  float gi_min_dist2;             /* SSGI squared-distance clamp */
  const float* kernel;            /* host, samples x 4 floats: tangent-frame hemisphere kernel; copied */
  int blocker_samples;            /* PCSS blocker-search taps, <= MRR_MAX_TAPS */
  int pcf_samples;                /* PCSS filter taps, <= MRR_MAX_TAPS */
  const float* blocker_taps;      /* host, blocker_samples x 2 floats in the unit disk; copied */
  const float* pcf_taps;          /* host, pcf_samples x 2 floats in the unit disk; copied */
  float light_size;               /* side of the square area light (world units) */
  float shadow_bias;              /* light-depth bias */
  int max_width, max_height;      /* largest frame mrr_render / mrr_masks will see (sizes pools) */
  /* tuning knobs (0 = library default); they change speed, never results */
  int lanes_per_texel;            /* SSAO work-list kernel: lanes sharing one texel's samples: 1, 2 or 4
                                     (default 1; with 64 samples and 1 lane the kernel compiled for that
                                     count runs) */
  int lanes_per_pixel;            /* SSAO full-resolution kernel: lanes sharing one pixel: 1, 2 or 4
                                     (default 1, likewise) */
  int no_graph;                   /* 1: mrr_render launches its kernels one by one instead of replaying a
                                     CUDA graph of them (the graph is re-captured whenever the frame
                                     descriptor or output pointer changes) */
  /* Sec. 4.1: bilateral blur of rendered sub-images (see mrr_blur_level); off when all 0 */
  int blur[MRR_MAX_LEVELS];       /* 1: mrr_render blurs level i's sub-image before the blend; only
                                     enabled levels i >= 1 (level 0 is the full-resolution image) */
  float blur_depth_rel;           /* the blur's depth test: |d' - d| <= blur_depth_rel * d; >= 0, finite */
  int merge_mode;                 /* 0: direct upsampling of every level (Sec. 4.2); 1: step-wise
                                     chain (Sec. 3.3), see mrr_upsample_merge; 2: direct upsampling
                                     with bilateral taps (Sec. 3.3), see mrr_upsample_merge_bilateral */
  int sample_levels;              /* 1: sample-count levels (Sec. 6): levels above 0 are rendered at full
                                     resolution with fewer samples instead of at a lower resolution (see
                                     mrr_shade_level); requires blur all 0 and merge_mode 0 */
  int pyramid_gathers;            /* 1 (SSAO only, not with sample_levels): the depth gathers of levels
                                     above 0 read the level's point samples -- the depth at s_i(Q) of
                                     the level-i block Q the projected pixel lies in -- instead of the
                                     full-resolution pixel (a point-sampled depth pyramid, built in the
                                     context's pools: frames up to the max size).  Single-frame calls
                                     only: batches and servers return MRR_EUNSUPPORTED */
  int disjoint;                   /* 1: complementary tiles without overlap -- the decomposition Sec. 3.1
                                     describes and rejects, built as an ablation.  Level i keeps only the
                                     blocks of its own mask of which no finer enabled level renders any
                                     pixel (no nesting; the coarsest level too), so no area is rendered
                                     twice; a pixel that no level covers is a "dead pixel".  The
                                     recomposition takes each pixel from its finest covering level,
                                     interpolated over that level's rendered texels only, with no
                                     blending; dead pixels (and pixels whose covering level has no
                                     rendered tap of positive weight) are NaN, and their label is 255.
                                     Requires blur all 0, merge_mode 0, sample_levels 0 and
                                     pyramid_gathers 0; single-frame calls only (batches and servers
                                     return MRR_EUNSUPPORTED) */
} mrr_config;

/* A pinhole camera: world-space eye and orthonormal basis (right, up, forward), the
 * tangent of half the vertical field of view, near and far.  View space is
 * (right, up, -forward).  Linear depth is the distance along forward.  The frame's camera
 * must satisfy 2^-60 <= near_plane < far_plane <= 2^60 (MRR_EINVAL otherwise). */
typedef struct mrr_camera {
  float eye[3], right[3], up[3], forward[3];
  float tan_half_fov, near_plane, far_plane;
} mrr_camera;

/* One frame's G-buffer (Sec. 3.1: "the information available in the G-Buffer"). */
typedef struct mrr_gbuffer {
  int width, height;
  const float* depth;       /* device [H][W] linear view depth; sky pixels hold cam.far_plane */
  const void* normal;       /* device [H][W] view-space unit normal: float4 (FP32) / half4 (FP16) */
  const void* color;        /* device [H][W] half4 direct light (SSGI only; else may be NULL) */
  const void* shadow_map;   /* device [S][S] linear light depth: float (FP32) / half (FP16); SSM only */
  int shadow_size;          /* S */
  mrr_camera cam;
  mrr_camera light;         /* SSM only: the light's camera (square frustum) */
} mrr_gbuffer;

/* Per-level mask buffers (caller-owned device memory), written by mrr_masks. */
typedef struct mrr_levels {
  int num_levels;                       /* must equal the context's num_levels */
  int width[MRR_MAX_LEVELS];            /* W_i (width[0] = W) */
  int height[MRR_MAX_LEVELS];           /* H_i */
  float* alpha[MRR_MAX_LEVELS];         /* [H_i][W_i] blurred mask a_i in [0,1] */
  uint8_t* stencil[MRR_MAX_LEVELS];     /* [H_i][W_i] S_i in {0,1} */
  uint32_t* worklist[MRR_MAX_LEVELS];   /* capacity W_i*H_i entries (y << 16) | x, row-major */
  uint32_t* counts;                     /* [MRR_MAX_LEVELS] entries written per list (device) */
  uint8_t* label;                       /* [H][W] owning level of each pixel, or NULL */
} mrr_levels;

typedef struct mrr_ctx mrr_ctx;

/* Level dimensions (pure helper, no context): W_i = ceil(W/2^i), H_i = ceil(H/2^i).
 * MRR_EINVAL for W or H outside [1, 16384] or level outside [0, MRR_MAX_LEVELS). */
mrr_status mrr_level_dims(int width, int height, int level, int* level_width, int* level_height);

/* Create a context: validates cfg, copies its sample tables (hemisphere kernel,
 * disk taps) and computes the Gaussian weights of each level (Sec. 3.1, Table 1):
 * radius R_i = ceil(3 sigma_i), weights exp(-k^2 / (2 sigma_i^2)) normalised over
 * [-R_i, R_i] in double and rounded to float.  Allocates the device pools that
 * mrr_render uses for frames up to max_width x max_height on the current device.
 * *out receives the context (NULL on failure). */
mrr_status mrr_create(const mrr_config* cfg, mrr_ctx** out);

/* Free the context and its pools.  The caller must ensure no work using them is
 * still in flight (synchronise the streams it used).  NULL is ignored. */
void mrr_destroy(mrr_ctx* ctx);

/* Sec. 3.1: the edge image.  edges_dev [H][W] gets 1 at a non-sky pixel that
 *  (a) has a sky 4-neighbour, or (b) whose second difference of depth along x or y
 *  exceeds depth_rel * depth (an axis counts only with both neighbours in the image),
 *  or (c) whose normal's dot product with an in-image non-sky 4-neighbour's is below
 *  normal_cos (first derivative of the normals), or (d) for MRR_SSM, whose one-sample
 *  hard shadow differs from an in-image non-sky 4-neighbour's; else 0.  Sky pixels
 *  are 0.  Edge maps are combined by maximum (Sec. 3.1).  For MRR_SSM frames up to the
 *  context's max size the hard shadows pass through a scratch pool of the context, so
 *  such calls on one context must not overlap on different streams. */
mrr_status mrr_edges(mrr_ctx* ctx, const mrr_gbuffer* g, uint8_t* edges_dev, void* stream);

/* Sec. 3.1 + Sec. 4.1: the masks of every level from the edge image [H][W] with
 * W = lv->width[0], H = lv->height[0] (at most the context's max size).  For each
 * enabled level i below the coarsest: D_i = maximum of the edge image over each
 * texel's block, a_i = Gaussian blur of D_i (sigma_i^2, horizontal then vertical, zero
 * outside the level), S_i = [a_i > 0] OR-ed with every set texel of the previous
 * enabled finer level inside the block (inclusive nesting, Fig. 2/3).  The coarsest
 * level has a = 1, S = 1; disabled levels a = 0, S = 0.  Then the work lists: the
 * texels with S_i = 1 in row-major order, counts[i] = their number (left on the
 * device), and label[p] = the finest enabled level whose stencil covers p. */
mrr_status mrr_masks(mrr_ctx* ctx, const uint8_t* edges_dev, const mrr_levels* lv, void* stream);

/* Sec. 3.2 / Sec. 4.1: render sub-image `level` only where its mask allows: for every
 * texel q in lv->worklist[level] (count lv->counts[level], read on the device),
 * c_level_dev[q] = the context's effect evaluated at full-resolution pixel s_i(q)
 * from the full-resolution G-buffer.  Other texels are not written.  c_level_dev is
 * [H_i][W_i] of float (FP32) / half (FP16), 4 per texel (rgb + 0) for MRR_SSGI.
 * With cfg.sample_levels = 1 and level > 0 (Sec. 6), c_level_dev is [H][W] instead: every
 * full-resolution pixel p of each listed texel's block [2^i q, 2^i q + 2^i) gets the
 * effect at p computed with every 2^i-th entry of each sample table (entries 0, 2^i,
 * 2 2^i, ...: ceil(n / 2^i) of n hemisphere samples, blocker taps and filter taps). */
mrr_status mrr_shade_level(mrr_ctx* ctx, int level, const mrr_gbuffer* g, const mrr_levels* lv,
                           void* c_level_dev, void* stream);

/* mrr_shade_level for every enabled level in ONE launch (the launch mrr_render makes):
 * a persistent grid strides over the concatenated work lists, whose lengths it reads
 * from lv->counts on the device.  c_levels_dev[i] as in mrr_shade_level (NULL for
 * disabled levels). */
mrr_status mrr_shade_levels(mrr_ctx* ctx, const mrr_gbuffer* g, const mrr_levels* lv, void* const* c_levels_dev,
                            void* stream);

/* Sec. 4.1: bilateral blur of sub-image `level` (1 <= level < num_levels, enabled).
 * The paper blurs the SSAO sub-images, above all the coarse ones, against the effect's
 * variance, without taking values from unrendered texels.  For every texel q with
 * lv->stencil[level][q] = 1:
 *   b_level_dev[q] = sum_t w_t c(q + t) / sum_t w_t
 * over the offsets t = (tx, ty), tx, ty in -2..2, whose texel q + t is inside the level,
 * has its stencil set, and passes the depth test
 *   |d(s_i(q + t)) - d(s_i(q))| <= cfg.blur_depth_rel * d(s_i(q))
 * (d = g->depth at a texel's sample pixel); w_t = B[tx] B[ty], B = (1, 4, 6, 4, 1).
 * q itself always passes, so the weight sum is at least 36.  Sums in row-major window
 * order, each operation one IEEE float operation; FP16 sub-images are read as half and
 * the quotient rounded to half.  Texels whose stencil is 0 are neither read nor written
 * (lv->worklist and lv->counts are not used).  c_level_dev and b_level_dev are laid out
 * as in mrr_shade_level and must be distinct buffers (MRR_EINVAL otherwise). */
mrr_status mrr_blur_level(mrr_ctx* ctx, int level, const mrr_gbuffer* g, const mrr_levels* lv,
                          const void* c_level_dev, void* b_level_dev, void* stream);

/* Sec. 4.2 and Eq. (1): upsample every enabled sub-image to full resolution and blend
 * them from the coarsest to the finest: a_i is interpolated bilinearly, c_i bilinearly
 * over rendered taps only (weights renormalised), alpha = min(w_i a_i, 1) and
 * c' = c_i alpha + c' (1 - alpha), starting from c' = the coarsest sub-image.
 * With cfg.merge_mode = 1, the step-wise reading of Sec. 3.3 instead: starting from the
 * coarsest sub-image, each finer enabled level i is blended at its own resolution with
 * the previous composite scaled up to it (plain bilinear; texel q of level i sits at
 * (2^i q + o_i - o_j) / 2^j in texels of the previous level j, taps clamped):
 * comp_i(q) = c_i(q) alpha + up (1 - alpha), alpha = min(w_i a_i(q), 1), where
 * S_i(q) = 1 and alpha > 0, else up; the output is the composite at level 0.  That mode
 * keeps the intermediate composites in the context's pools, so the frame must fit the
 * context's max size (MRR_EINVAL otherwise).
 * With cfg.sample_levels = 1 every c_levels_dev[i] is [H][W] and only the masks are
 * interpolated: per pixel, from c' = c_{L-1}(p), each finer enabled level i whose texel
 * (p_x >> i, p_y >> i) is rendered blends in c_i(p) with alpha = min(w_i a_i(p), 1), a_i
 * interpolated as above.
 * c_levels_dev[i] as in mrr_shade_level (NULL for disabled levels).  out_dev is
 * [H][W] float, or [H][W] float4 (rgb + 0) for MRR_SSGI. */
mrr_status mrr_upsample_merge(mrr_ctx* ctx, const mrr_levels* lv, void* const* c_levels_dev, float* out_dev,
                              void* stream);

/* Sec. 3.3 (bilateral upsampling, after Tomasi and Manduchi): mrr_upsample_merge for a
 * context with cfg.merge_mode = 2, which needs the frame's depth (g->depth; the other
 * planes of g are not read).  As the direct merge, except that c_i is interpolated over
 * the rendered taps Q whose sample depth lies on the pixel's surface,
 *   |d(s_i(Q)) - d(p)| <= cfg.blur_depth_rel * d(p),
 * and over every rendered tap when none does; a_i stays plain bilinear.  mrr_upsample_merge
 * itself returns MRR_EINVAL for such a context; mrr_render passes the depth itself. */
mrr_status mrr_upsample_merge_bilateral(mrr_ctx* ctx, const mrr_gbuffer* g, const mrr_levels* lv,
                                        void* const* c_levels_dev, float* out_dev, void* stream);

/* The whole method for one frame on one stream: edges, masks, work lists, all
 * sub-images, the blur of the levels cfg.blur names, blend -- using the context's pools
 * for every intermediate.  Frames up to
 * the context's max size.  out_dev as in mrr_upsample_merge. */
mrr_status mrr_render(mrr_ctx* ctx, const mrr_gbuffer* g, float* out_dev, void* stream);

/* Tracing hook (an addition for measurement): with two CUDA events (cudaEvent_t passed
 * as void*, created with timing), every following mrr_render records event_begin on its
 * stream immediately before the work-list shading launch of the frame path and event_end
 * immediately after it, so cudaEventElapsedTime gives that launch's device time inside a
 * real frame; while set, mrr_render launches its kernels one by one instead of replaying
 * a CUDA graph.  The caller keeps the events alive until tracing ends.  NULL, NULL ends
 * tracing.  MRR_EINVAL if exactly one event is NULL. */
mrr_status mrr_trace_shading(mrr_ctx* ctx, void* event_begin, void* event_end);

/* Naive full-resolution rendering (the paper's comparison, Sec. 5): the effect at
 * every pixel.  out_dev as in mrr_upsample_merge. */
mrr_status mrr_render_full(mrr_ctx* ctx, const mrr_gbuffer* g, float* out_dev, void* stream);

/* mrr_render from host memory: copies the G-buffer planes named by g (host pointers,
 * pinned for full speed) into the context's device pools on `stream`, renders, copies
 * the result to out_host and synchronises the stream before returning. */
mrr_status mrr_render_host(mrr_ctx* ctx, const mrr_gbuffer* g_host, float* out_host, void* stream);

/* mrr_render_host for a stream of frames: the same copies and rendering, enqueued on the
 * context's own streams and not waited for.  Consecutive calls use two device input /
 * output sets in turn, so one frame's host-to-device copy overlaps the previous frame's
 * rendering and device-to-host copy (renders themselves run one after another).  The
 * host planes named by g_host and out_host (pinned for full speed) must stay valid, and
 * the inputs unmodified, until mrr_render_host_wait returns; out_host holds the image
 * after it.  Not thread-safe on one context. */
mrr_status mrr_render_host_async(mrr_ctx* ctx, const mrr_gbuffer* g_host, float* out_host);

/* Waits for every frame mrr_render_host_async has enqueued on the context. */
mrr_status mrr_render_host_wait(mrr_ctx* ctx);

/* mrr_masks for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the mask stage.  Host programs that may
 * not call cudaMalloc (a plug-in inside an engine that owns every device allocation, a
 * process working inside a pre-reserved memory budget) cannot create a context, since
 * mrr_create allocates pools.  This call needs no context: it reads only the mask fields
 * of *cfg (num_levels, sigma2, enabled, force_level0; host memory), computes exactly
 * what mrr_masks computes into the caller's buffers, and keeps its one piece of scratch
 * -- the work-list compaction's per-chunk counts -- in a fixed 32 KiB array that the
 * library holds on every device that loads it until the process exits.
 *  - Frames up to 4096 x 4096 pixels; larger frames (or inconsistent level sizes or
 *    missing buffers) return MRR_EINVAL before anything is launched.
 *  - It allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *  - The first call on each device looks the array's device address up (with that
 *    device current) and keeps it; make that first call before any stream capture.
 *    Under lazy module loading (CUDA's default) that first lookup may also make the
 *    driver load this library's device code, which reserves device memory once; a
 *    caller with a strict budget should make the first call during its own set-up.
 *    The kept address belongs to the device's primary context: after a
 *    cudaDeviceReset in the same process it is stale, so do not call this again then.
 *  - Every call shares the array: calls that overlap on the GPU (other streams, other
 *    host threads) race on it; order them.  Returns MRR_ECUDA on a launch failure. */
mrr_status mrr_masks_static(const mrr_config* cfg, const uint8_t* edges_dev, const mrr_levels* lv, void* stream);

/* Result of mrr_autotune: the settings chosen and the measured kernel times (ms). */
typedef struct mrr_tuning {
  int lanes_per_texel;      /* chosen split of a work-list texel's samples over lanes */
  int grid_multiplier;      /* work-list kernel grid = multiplier x (SMs x resident CTAs per SM) */
  int lanes_per_pixel;      /* chosen split for the full-resolution kernel */
  float shade_levels_ms;    /* work-list shading kernel time with the chosen settings */
  float shade_full_ms;      /* full-resolution kernel time with the chosen setting */
  int candidates;           /* configurations timed */
} mrr_tuning;

/* Autotuner: times every supported (lanes_per_texel, grid_multiplier) pair of the
 * work-list shading kernel and every lanes_per_pixel of the full-resolution kernel on
 * this frame (median of 5 timed launches after 2 warm-up launches each, CUDA events on
 * `stream`), keeps the fastest in the context (they change speed, never results) and
 * reports them in *out (may be NULL).  Runs mrr_edges / mrr_masks into the context's
 * pools first; synchronises `stream`.  Settings fixed in the config (non-zero
 * lanes_per_texel / lanes_per_pixel) are kept. */
mrr_status mrr_autotune(mrr_ctx* ctx, const mrr_gbuffer* g, void* stream, mrr_tuning* out);

/* Batched rendering: several frames -- of different sizes, through different contexts
 * and so possibly different effects and precisions -- in one pass, with ONE persistent
 * shading launch for all of them.  That launch pulls fixed-size chunks of the
 * concatenated work lists of every frame and level from a global queue (an atomic
 * counter), so cheap and expensive frames balance across the GPU.  Edges, masks and
 * the blend run per frame as in mrr_render; every frame's image equals mrr_render of the
 * same context and frame, bit for bit.  The paper renders one frame at a time; this is
 * a serving extension of its Sec. 3 pipeline. */
typedef struct mrr_batch mrr_batch;

/* Tuning of a batch (0 = default): entries per queue chunk (multiple of 32, at most
 * 65536) and the launch grid as a multiple of the resident CTAs. */
typedef struct mrr_batch_tuning {
  int chunk;
  int grid_multiplier;
  float shade_ms;       /* batched shading launch time with these settings (autotune output) */
  int candidates;       /* configurations timed (autotune output) */
} mrr_batch_tuning;

/* Create a batch object: device item table for up to 8 frames, queue head, pinned
 * staging.  Allocates; not for capture. */
mrr_status mrr_batch_create(mrr_batch** out);
void mrr_batch_destroy(mrr_batch* b);

/* Render frames[k] through ctxs[k] into outs[k] (as mrr_render), k < n <= 8, on one
 * stream.  The contexts must be distinct (each frame uses its context's pools) and each
 * frame must fit its context.  Replays a CUDA graph of the batch while the contexts,
 * frame descriptors and outputs repeat. */
mrr_status mrr_render_batch(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, float* const* outs, int n,
                            void* stream);

/* Text of the batch's last failure ("" if none). */
const char* mrr_batch_last_error(mrr_batch* b);

/* Autotuner of the batched launch: times chunk in {256, 1024, 4096} x grid_multiplier in
 * {1, 2} (median of 5 after 2 warm-ups, CUDA events on `stream`), keeps the fastest in
 * the batch and reports it in *out (may be NULL).  Synchronises `stream`. */
mrr_status mrr_batch_autotune(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, int n, void* stream,
                              mrr_batch_tuning* out);

/* Serving.  A server renders a stream of frame requests of mixed size and effect.  It
 * keeps `slots` sets of device state resident (one context per enabled effect -- level
 * pyramids, work lists, sub-images -- plus a stream and a batch object each); fewer if
 * creating the next set would leave less than hbm_reserve bytes of free device memory.
 * A scheduler thread admits pending requests in arrival order as slots free up, packs
 * up to per_effect requests of each effect into one batch (one persistent shading launch,
 * see mrr_render_batch; a slot holds per_effect contexts per effect) and overlaps batches
 * on the slots' streams.  A batch runs as a CUDA graph keyed on its topology -- which
 * contexts, in a fixed order -- not on its buffers: each batch is captured afresh and
 * applied to the cached graph of its topology with cudaGraphExecUpdate, and only a
 * topology not seen before is instantiated (mrr_server_stats counts both).  Every result
 * equals mrr_render of the same frame with the same configuration.  The paper renders
 * frames one by one; this is the serving extension of its Sec. 3 pipeline. */
typedef struct mrr_server mrr_server;

typedef struct mrr_server_config {
  mrr_config effect_cfg[3];   /* per effect, indexed by mrr_effect; max_width / max_height = the
                                 largest frame served with that effect; the tables are copied */
  int effect_enabled[3];      /* effects this server accepts */
  int slots;                  /* batches in flight at most (0 = 4) */
  size_t hbm_reserve;         /* free device memory (bytes) slot creation must leave untouched */
  int max_queue;              /* pending requests beyond which mrr_submit returns MRR_EBUSY (0 = 1024) */
  int mock_device_us;         /* test mode: no device work at all; a batch completes after this many
                                 microseconds of host time (scheduler tests without a GPU) */
  int per_effect;             /* requests of one effect a batch may hold (0 = 2); at most 8 requests in
                                 all: per_effect * enabled effects <= 8, else MRR_EINVAL */
  int direct_launches;        /* 1: batches launched kernel by kernel, without graphs */
} mrr_server_config;

typedef struct mrr_request {
  mrr_effect effect;
  mrr_gbuffer frame;          /* device pointers; must stay valid until the request completes */
  float* out_dev;             /* output as for mrr_render; written when the request completes */
} mrr_request;

typedef struct mrr_request_info_t {
  int done;
  mrr_status result;
  int64_t submit_ns, start_ns, done_ns;  /* host steady clock: submitted, dispatched, completed */
  float device_ms;                       /* device time of the batch the request ran in */
} mrr_request_info_t;

/* Create a server on the current device (allocates its slots); MRR_ENOMEM if not even
 * one slot fits.  mrr_server_slots reports how many were created. */
mrr_status mrr_server_create(const mrr_server_config* cfg, mrr_server** out);
int mrr_server_slots(mrr_server* s);
/* Stop the scheduler, wait for work in flight, free everything. */
void mrr_server_destroy(mrr_server* s);

/* Queue a request; *ticket identifies it.  MRR_EINVAL for an effect the server does not
 * serve or a frame larger than its context allows; MRR_EBUSY when max_queue requests
 * are already pending.  Thread-safe. */
mrr_status mrr_submit(mrr_server* s, const mrr_request* r, uint64_t* ticket);
/* Non-blocking: *done = 1 once the request has completed; *result its status. */
mrr_status mrr_poll(mrr_server* s, uint64_t ticket, int* done, mrr_status* result);
/* Block until the request completes (its status is returned) or timeout_ns elapses
 * (MRR_ETIMEDOUT); timeout_ns < 0 waits without limit. */
mrr_status mrr_wait(mrr_server* s, uint64_t ticket, int64_t timeout_ns);
/* Timing record of a request (valid until mrr_release). */
mrr_status mrr_request_info(mrr_server* s, uint64_t ticket, mrr_request_info_t* out);
/* Forget a completed request's record. */
mrr_status mrr_release(mrr_server* s, uint64_t ticket);

typedef struct mrr_server_stats_t {
  uint64_t batches;               /* batches dispatched */
  uint64_t completed;             /* requests completed */
  uint64_t graph_instantiations;  /* batch graphs instantiated (a topology not cached) */
  uint64_t graph_updates;         /* batch graphs updated in place (a cached topology) */
} mrr_server_stats_t;

/* Counters of the server's scheduler since it was created.  Thread-safe. */
mrr_status mrr_server_stats(mrr_server* s, mrr_server_stats_t* out);

/* Number of kernels this library has launched in this process (all contexts), for
 * accounting of GPU work in benchmarks. */
uint64_t mrr_kernel_launches(void);

/* Text of the last failure on this context ("" if none); valid until the next call. */
const char* mrr_last_error(mrr_ctx* ctx);

/* Device-side fault bits of the context: kernels that wait on asynchronous tile loads
 * give up after about a second and record a bit here instead of waiting for ever (bit 0:
 * edge detection; bit 30: mrr_check_wait_timeout); the output of a frame whose edge
 * loads gave up is invalid.  Synchronises the device, copies the word to *flags and, if
 * `clear` is nonzero, resets it.  Not part of the paper's method; it makes a stalled load
 * visible to the host. */
mrr_status mrr_fault_flags(mrr_ctx* ctx, uint32_t* flags, int clear);

/* Self-check of that failure path: runs one CTA that waits, with the edge kernel's
 * bounded wait, on an mbarrier phase that expects 16 bytes of transactions no copy will
 * ever bring.  The wait gives up after about a second of SM clocks, the kernel records
 * bit 30 in the context's fault word and returns -- no fault, no hang, the context stays
 * usable.  Synchronises the device before and after; copies the fault word (not cleared)
 * to *flags.  Takes about one second. */
mrr_status mrr_check_wait_timeout(mrr_ctx* ctx, uint32_t* flags);

/* Diagnostic: the effect kernels project sample points with their own correctly rounded
 * reciprocal (Newton-Raphson refinement of the hardware estimate) instead of IEEE
 * division.  This runs it over every float whose bit pattern lies in [first_bits,
 * last_bits], and over their negatives, on the current device, compares each result bit
 * for bit with IEEE division and stores the number of differences in *mismatches (0 over
 * [2^-64, 2^64) is the claim the projections rely on).  Synchronous; allocates 8 bytes
 * of device memory for the count.  MRR_EINVAL for a NULL pointer or last < first.  Not
 * part of the paper's method. */
mrr_status mrr_check_reciprocal(uint32_t first_bits, uint32_t last_bits, uint64_t* mismatches);

#ifdef __cplusplus
}
#endif

#endif /* MRR_H */
