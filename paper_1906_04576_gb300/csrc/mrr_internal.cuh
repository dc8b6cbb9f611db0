// mrr_internal.cuh -- device-side parameter blocks and kernel launchers of libmrr.
//
// Every kernel is compiled with -fmad=false and IEEE division / square root, so each
// floating-point operation is one correctly rounded IEEE operation in the order the
// source writes it.  The order of every expression below is part of the method's
// definition (it decides which samples are occluded), so it must not be "simplified".
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/mrr.h"

namespace mrr {

// half4: four binary16 values, 8-byte aligned (FP16 normals, SSGI colour, FP16 SSGI
// sub-images).
struct __align__(8) half4 {
  __half x, y, z, w;
};

// Pinhole constants of the viewing camera, derived in double on the host from the
// frame's float camera and rounded once to float (see make_view in api.cu):
//   slope_x(x) = (x + 1/2) ax - bx,  slope_y(y) = by - (y + 1/2) ay,
//   pixel X = (u + bx) kx,  Y = (by - v) ky  for a view direction (u, v, -1).
struct ViewC {
  int W, H;
  float ax, bx, kx, ay, by, ky, nearp, farp;
};

// World-space basis of the viewing camera and the light camera (soft shadows).
struct LightC {
  float ce[3], cr[3], cu[3], cf[3];  // viewing camera eye / right / up / forward
  float le[3], lr[3], lu[3], lf[3];  // light camera
  float tl, kl, nearp, farp;         // light tan(half fov), S / (2 tl), near, far
  int S;                             // shadow map side
};

// Everything an effect needs, passed by value as a kernel parameter so the sample
// tables are read through the constant cache (every lane of a warp reads the same
// sample at the same time).
struct ShadeParams {
  int effect;
  ViewC v;
  LightC L;
  int samples;
  float radius, ao_bias, gi_min_dist2;
  float light_half, shadow_bias;
  int nb, np;
  float4 kernel[MRR_MAX_SAMPLES];                  // (x, y, z, 0) per sample
  float kx[MRR_MAX_SAMPLES], ky[MRR_MAX_SAMPLES], kz[MRR_MAX_SAMPLES];  // the same, split for paired loads
  float2 btaps[MRR_MAX_TAPS];
  float2 ptaps[MRR_MAX_TAPS];
};

// Frame inputs (device pointers).
struct FrameIn {
  const float* depth;
  const void* normal;  // float4 or half4
  const half4* color;  // SSGI
  const void* smap;    // float or half
};

struct EdgeParams {
  ViewC v;
  LightC L;
  float depth_rel, normal_cos, shadow_bias;
  int ssm;
  uint32_t* fault;  // device fault word of the context (tma.cuh)
  uint32_t* zero;   // words the launch sets to 0 for the next kernel (may be null)
  int zero_words;
  uint32_t* ebits;  // non-null: write the edge image bit-packed here, ewords words per row
  int ewords;
  // soft shadows: scratch for the one-sample hard shadows as bits (ewords words per row).
  // Non-null lets a frame whose rows allow TMA take the two-pass path (shadow bits, then
  // the TMA edge kernel); null keeps the one-pass staged kernel.
  uint32_t* sbits;
  // 1: the frame is one of a batch or a served stream, whose kernels share the SMs with
  // other streams' kernels (selects the edge kernel's form that does better there)
  int concurrent;
};

// Mask stage of all levels in one launch (k_masks.cu).  Level i: mode 0 = blur,
// 1 = all ones (coarsest level or forced level 0), 2 = all zero (disabled).
constexpr int MASK_TILE = 32;    // full-resolution pixels per CTA tile side
constexpr int MASK_MARGIN = 24;  // halo of the staged edge image: max R_i 2^i over blurred levels
struct MaskParams {
  int W, H, L;
  int mode[MRR_MAX_LEVELS];
  int R[MRR_MAX_LEVELS];
  float g[MRR_MAX_LEVELS][16];   // Gaussian taps k = -R..R
  int Wi[MRR_MAX_LEVELS], Hi[MRR_MAX_LEVELS];
  float* alpha[MRR_MAX_LEVELS];
  uint8_t* stencil[MRR_MAX_LEVELS];
  uint8_t* label;                // [H][W] or null
  // level 0's horizontal blur as a table: lut0[b] = the ascending-tap sum of g over the
  // set bits of the (2R+1)-bit window b (null: sum the taps directly; any R <= 6)
  const float* lut0;
  // levels >= 1: the same tables for their radii, read from global memory (null: sum the
  // taps directly; R <= MASK_LUT_GLOBAL_R)
  const float* lut[MRR_MAX_LEVELS];
  // Frame mode (a0c non-null): the kernel also writes every enabled level's work list
  // (tiles in any order, texels of a tile in row-major order), level 0's a only as a0c
  // (aligned with level 0's list), and neither alpha[0] nor stencil[0].
  float* a0c;
  const uint32_t* ebits;  // non-null: the edge image bit-packed (ewords words per row), read instead of E
  int ewords;
  uint32_t* list[MRR_MAX_LEVELS];
  uint32_t* counts;  // entries per level, zero before the launch (the tiles add to it)
  int disjoint;      // complementary tiles without overlap (the variant Sec. 3.1 rejects)
  // Frame mode, level 0 blurred: the Chebyshev radius r1 within which any one edge pixel
  // already makes min(w_0 a_0, 1) = 1 (-1: none).  a_0 is a fused multiply-add chain of
  // non-negative terms, so it is at least fl(g[R+dy] g[R+dx]) for an edge at (dx, dy), and
  // fl(w_0 a_0) >= 1 wherever fl(w_0 fl(g[R+dy] g[R+dx])) >= 1 for every offset of the
  // box; there a0c holds 1, which the level-0 blend turns into the same alpha of 1.
  int sure0;
};
constexpr int MASK_LUT_MAX = 512;  // level 0's table for R <= 4 (larger R sums the taps)

// The truncated Gaussian of Sec. 3.1 / Table 1: R = ceil(3 sigma), weights
// exp(-k^2 / (2 sigma^2)) normalised over [-R, R] in double (ascending k), rounded once to
// float.  Returns R (0 when sigma2 <= 0).
int mask_gauss(double sigma2, float* g);

// Fills the parts of a MaskParams that follow from the configuration and the level
// buffers: sizes, per-level mode (0 blur, 1 all ones, 2 disabled), radius and taps, the
// output planes and the label plane.  Returns false when a
// blurred level has sigma2 <= 0 or a radius above 6.
bool mask_level_params(const mrr_config& c, const mrr_levels* lv, MaskParams& m);
constexpr int MASK_LUT_GLOBAL_R = 6;  // tables of the levels above 0 up to 2^13 entries

// Work-list compaction of all levels in one launch: level l owns chunks
// [chunk_begin[l], chunk_begin[l+1]) of COMPACT_CHUNK texels each.
constexpr int COMPACT_CHUNK = 4096;
constexpr int COMPACT_THREADS = 256;
struct CompactParams {
  int nlev;
  int level_of[MRR_MAX_LEVELS];          // which level slot l refers to
  int chunk_begin[MRR_MAX_LEVELS + 1];
  int Wi[MRR_MAX_LEVELS], Hi[MRR_MAX_LEVELS];
  const uint8_t* stencil[MRR_MAX_LEVELS];
  uint32_t* list[MRR_MAX_LEVELS];
  uint32_t* chunk_counts;                // [chunk_begin[nlev]]
  uint32_t* counts;                      // [MRR_MAX_LEVELS]
  int zero_mask;                         // bit i: counts[i] = 0 (levels not compacted)
};

// Shading of all listed texels of several levels in one launch.
struct ShadeLevels {
  int nlev;
  int level[MRR_MAX_LEVELS];
  const uint32_t* list[MRR_MAX_LEVELS];
  void* c[MRR_MAX_LEVELS];
  int Wi[MRR_MAX_LEVELS], Hi[MRR_MAX_LEVELS];
  const uint32_t* counts;  // device, indexed by level; clamped to W_i * H_i when read
  // bit k set: slot k stores its values at the entry's list position (a list-aligned,
  // compact sub-image) instead of at texel (qy, qx)
  int compact;
  // pyramid gathers (SSAO): slot k's depth gathers read pyr[k], the level's point-sampled
  // depth ([H_i][W_i], depth at s_i(Q)); null for level 0, which reads full resolution
  int pyramid;
  const float* pyr[MRR_MAX_LEVELS];
};

// Point-sampled depth of levels above 0 for pyramid gathers (k_shade.cu): slot k writes
// out[k][Q] = depth[s_i(Q)] for every texel Q of level level[k].
struct PyramidParams {
  int W, H, nlev;
  const float* depth;
  int level[MRR_MAX_LEVELS];
  int Wi[MRR_MAX_LEVELS], Hi[MRR_MAX_LEVELS];
  float* out[MRR_MAX_LEVELS];
};

// One sample-count level (Sec. 6): every full-resolution pixel of each listed texel's
// block [2^level q, 2^level q + 2^level) is shaded into the [H][W] sub-image c.
struct BlockLevel {
  int level, Wi, Hi;
  const uint32_t* list;
  const uint32_t* count;  // device: entries in the list (clamped to W_i * H_i when read)
  void* c;
};

// One frame of a batched shading launch (k_batch.cu); an array of these lives in
// device memory.
constexpr int MAX_BATCH = 8;
struct BatchItem {
  ShadeParams p;
  FrameIn in;
  ShadeLevels lv;
  int precision;
};

struct MergeParams {
  int W, H, L, C, half_store;
  int enabled[MRR_MAX_LEVELS];
  int Wi[MRR_MAX_LEVELS], Hi[MRR_MAX_LEVELS];
  float weight[MRR_MAX_LEVELS];
  const float* alpha[MRR_MAX_LEVELS];
  const uint8_t* stencil[MRR_MAX_LEVELS];
  const void* c[MRR_MAX_LEVELS];
};

// One step of the step-wise blending (Sec. 3.3, k_merge.cu): level i's composite dst
// ([H_i][W_i] float, float4 when C == 4) from the composite src of level j > i.
struct ChainParams {
  int C, half_store;
  int i, j;
  int Wi, Hi, Wj, Hj;
  float weight;            // w_i
  int blend;               // blend c_i in (level i enabled and its planes given)
  const float* alpha;      // a_i
  const uint8_t* stencil;  // S_i
  const void* c;           // c_i (sub-image storage type)
  const void* src;         // composite of level j, or the coarsest sub-image when src_sub
  int src_sub;
  float* dst;
};

// Level 0's part of Eq. (1) over level 0's work list, after the coarser levels are merged
// into `out`: entry k (pixel list[k]) has a_0 = a0c[k] and c_0 at position k of c0c.
struct Blend0Params {
  int W, H, C, half_store;
  float weight;
  const uint32_t* list;
  const uint32_t* count;  // device: entries in the list
  const float* a0c;
  const void* c0c;
};

// Bilateral blur of one or more levels' sub-images (k_blur.cu): slot k blurs every
// stencil texel of level `level[k]` from c[k] into b[k] (dense [H_i][W_i] sub-images);
// its tiles are blocks tile_begin[k] .. tile_begin[k + 1] - 1 of the launch.
struct BlurParams {
  int W, H, C, half_store;
  float rel;               // depth test: |d' - d| <= rel * d
  const float* depth;      // full-resolution depth
  int nlev;
  int level[MRR_MAX_LEVELS];
  int Wi[MRR_MAX_LEVELS], Hi[MRR_MAX_LEVELS];
  int tile_begin[MRR_MAX_LEVELS + 1];
  const uint8_t* stencil[MRR_MAX_LEVELS];
  const void* c[MRR_MAX_LEVELS];
  void* b[MRR_MAX_LEVELS];
};

// ---- launchers (return cudaGetLastError() of the launch)
cudaError_t launch_edges(const EdgeParams& p, const float* depth, const void* normal, int half_normal,
                         const float* smap, uint8_t* E, cudaStream_t s);
cudaError_t launch_masks(const MaskParams& m, const uint8_t* E, cudaStream_t s);
// The recomposition of the disjoint-tile ablation (k_merge.cu): each pixel from its finest
// covering level, no blending, NaN where no level covers it.
cudaError_t launch_merge_disjoint(const MergeParams& p, float* out, cudaStream_t s);
cudaError_t launch_compact(const CompactParams& p, cudaStream_t s);
cudaError_t launch_shade_levels(const ShadeParams& p, const FrameIn& in, int precision, const ShadeLevels& lv,
                                int grid, int split, cudaStream_t s);
cudaError_t launch_shade_full(const ShadeParams& p, const FrameIn& in, int precision, float* out, int split,
                              cudaStream_t s);
cudaError_t launch_shade_blocks(const ShadeParams& p, const FrameIn& in, int precision, const BlockLevel& b,
                                int grid_mult, cudaStream_t s);
cudaError_t launch_pyramid(const PyramidParams& p, cudaStream_t s);
cudaError_t launch_merge(const MergeParams& p, float* out, cudaStream_t s);
// bit patterns [first, last] as floats x: counts into *bad every x where the kernels'
// reciprocal of x or of -x differs from IEEE division
cudaError_t launch_check_reciprocal(uint32_t first, uint32_t last, unsigned long long* bad, cudaStream_t s);
cudaError_t launch_blend0(const Blend0Params& p, float* out, cudaStream_t s);
cudaError_t launch_chain(const ChainParams& p, cudaStream_t s);
// Blend of sample-count levels (every c[i] is [H][W]): the levels above 0, and level 0
// too where enabled[0] is set (full-resolution a_0, S_0, c_0).
cudaError_t launch_merge_samples(const MergeParams& p, float* out, cudaStream_t s);
// The direct merge with bilateral taps: c_i over the rendered taps whose sample depth is
// within rel * d(p) of the pixel's depth (all rendered taps when none is).
cudaError_t launch_merge_bilateral(const MergeParams& p, const float* depth, float rel, float* out, cudaStream_t s);
cudaError_t launch_blur(const BlurParams& p, cudaStream_t s);
// One CTA that waits, as the TMA edge kernel does, on an mbarrier phase nothing will
// complete, and records the timeout in *fault (tma.cuh's FAULT_CHECK_WAIT).
cudaError_t launch_check_wait(uint32_t* fault, cudaStream_t s);

void edges_prepare();     // one-time launch set-up of the edge kernels (before any stream capture)
int shade_grid_blocks();  // grid multiplier base of the work-list kernel (grid = multiple of its resident CTAs)
int batch_grid_blocks();  // resident CTAs of the batched shading kernel
int blur_tiles(int Wi, int Hi);  // blur tiles of a W_i x H_i level
cudaError_t launch_shade_batch(const BatchItem* items_dev, int nitems, uint32_t* queue_head, int chunk, int grid,
                               cudaStream_t s);

// Kernels launched by this library in this process (every launcher adds its launches).
std::atomic<uint64_t>& launch_counter();
inline void count_launches(int n) { launch_counter().fetch_add((uint64_t)n, std::memory_order_relaxed); }

}  // namespace mrr

// Serving uses the batch path without graph capture (api.cu).
mrr_status mrr_batch_enqueue_direct(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames,
                                    float* const* outs, int n, cudaStream_t stream);
// Serving: the batch as a CUDA graph keyed on its topology (contexts in order), captured
// afresh and applied to a cached graph of that topology with cudaGraphExecUpdate.
mrr_status mrr_batch_enqueue_graph(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames,
                                   float* const* outs, int n, cudaStream_t stream);
void mrr_batch_graph_counts(const mrr_batch* b, uint64_t* instantiations, uint64_t* updates);
