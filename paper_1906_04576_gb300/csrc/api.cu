// api.cu -- the C ABI of libmrr (include/mrr.h): argument validation, the host-side
// constants of each stage and the launches.  No exception crosses the ABI; every
// failure is a status code plus a message kept on the context.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mrr_internal.cuh"

using namespace mrr;

struct mrr_ctx {
  mrr_config cfg;
  float4 kernel[MRR_MAX_SAMPLES];
  float2 btaps[MRR_MAX_TAPS], ptaps[MRR_MAX_TAPS];
  float gauss[MRR_MAX_LEVELS][16];
  int R[MRR_MAX_LEVELS];
  int shade_grid = 0;
  int split_texel = 1, split_pixel = 1;  // SSAO lanes per texel / pixel
  std::string err;
  // pools of mrr_render / mrr_masks, sized for max_width x max_height
  int pool_W = 0, pool_H = 0;
  uint8_t* edges = nullptr;
  uint32_t* ebits = nullptr;  // mrr_render's bit-packed edge image
  uint32_t* sbits = nullptr;  // soft shadows: the one-sample hard shadows as bits (edge kernels' scratch)
  // mrr_trace_shading: events recorded around the frame path's shading launch
  cudaEvent_t trace_begin = nullptr, trace_end = nullptr;
  float* alpha[MRR_MAX_LEVELS] = {};
  uint8_t* stencil[MRR_MAX_LEVELS] = {};
  uint32_t* worklist[MRR_MAX_LEVELS] = {};
  void* cbuf[MRR_MAX_LEVELS] = {};
  void* bbuf[MRR_MAX_LEVELS] = {};  // blurred sub-images of the levels cfg.blur names
  float* comp[MRR_MAX_LEVELS] = {};  // step-wise blending's composites of levels 1 .. L-2
  float* pyr[MRR_MAX_LEVELS] = {};   // pyramid gathers: point-sampled depth of levels 1 .. L-1
  uint32_t* counts = nullptr;
  uint32_t* chunk_counts = nullptr;
  size_t chunk_cap = 0;
  float* lut0 = nullptr;  // level 0's horizontal blur table (device), see MaskParams
  float* lut[MRR_MAX_LEVELS] = {};  // the levels above 0's tables (device), see MaskParams
  uint32_t* fault = nullptr;  // device fault word (bits of tma.cuh)
  // pools of mrr_render_host
  float* h_depth = nullptr;
  void* h_normal = nullptr;
  void* h_color = nullptr;
  void* h_smap = nullptr;
  size_t h_smap_bytes = 0;
  float* h_out = nullptr;
  // mrr_render replays a CUDA graph of its launches while the frame's arguments repeat
  bool use_graph = true;
  // (two entries, so that frames alternating between two buffer sets both replay)
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec[2] = {};
  mrr_gbuffer graph_key[2];
  float* graph_out[2] = {};
  uint64_t graph_kernels[2] = {};
  int graph_next = 0;  // the entry a new capture replaces
  uint64_t graph_replays = 0;
  // mrr_render_host_async: two device input / output sets used in turn, and the streams
  // that overlap one frame's copies with the other's rendering
  struct HostSet {
    float* depth = nullptr;
    void* normal = nullptr;
    void* color = nullptr;
    void* smap = nullptr;
    size_t smap_bytes = 0;
    float* out = nullptr;
    bool used = false;
    cudaEvent_t loaded = nullptr, rendered = nullptr, done = nullptr;
  } hset[2];
  int hset_next = 0;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
};

struct mrr_batch {
  BatchItem* items_dev = nullptr;
  BatchItem* staging = nullptr;        // pinned host copy the item upload reads
  uint32_t* queue_head = nullptr;
  cudaEvent_t staging_done = nullptr;  // the last upload from `staging` has finished
  bool staging_pending = false;
  int chunk = 1024, grid_mult = 1;
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int key_n = 0;
  mrr_ctx* key_ctx[MAX_BATCH] = {};
  mrr_gbuffer key_frame[MAX_BATCH];
  float* key_out[MAX_BATCH] = {};
  int key_chunk = 0, key_grid = 0;
  uint64_t key_kernels = 0;
  // serving: graphs keyed on topology (the contexts, in order) rather than on pointers,
  // updated in place for every new set of frames (mrr_batch_enqueue_graph)
  struct TopoGraph {
    cudaGraphExec_t exec = nullptr;
    int n = 0, chunk = 0, grid = 0;
    mrr_ctx* ctx[MAX_BATCH] = {};
    uint64_t kernels = 0, last_use = 0;
  };
  static constexpr int TOPO_CACHE = 16;
  TopoGraph topo[TOPO_CACHE];
  uint64_t topo_clock = 0, graph_instantiations = 0, graph_updates = 0;
  std::string err;
};

namespace {

constexpr int MAX_DIM = 16384;
// camera depth range: every projected sample depth then lies where the kernels'
// reciprocal is the correctly rounded one (2^-64 <= d < 2^64)
constexpr float CAM_MIN_NEAR = 0x1p-60f, CAM_MAX_FAR = 0x1p60f;

mrr_status fail(mrr_ctx* ctx, mrr_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

#define MRR_CUDA(ctx, call)                                                                           \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail((ctx), MRR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

inline int level_dim(int n, int i) { return (n + (1 << i) - 1) >> i; }
inline int channels(const mrr_config& c) { return c.effect == MRR_SSGI ? 4 : 1; }
inline size_t cbytes(const mrr_config& c) {
  return (size_t)channels(c) * (c.precision == MRR_FP16 ? 2 : 4);
}
inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Pinhole constants in double from the float camera, rounded once to float:
// t_x = tan_half * (W / H); ax = 2 t_x / W, bx = t_x, kx = W / (2 t_x);
// ay = 2 tan_half / H, by = tan_half, ky = H / (2 tan_half).
ViewC make_view(int W, int H, const mrr_camera& c) {
  const double th = c.tan_half_fov;
  const double tx = th * ((double)W / (double)H);
  ViewC v;
  v.W = W;
  v.H = H;
  v.ax = (float)(2.0 * tx / (double)W);
  v.bx = (float)tx;
  v.kx = (float)((double)W / (2.0 * tx));
  v.ay = (float)(2.0 * th / (double)H);
  v.by = (float)th;
  v.ky = (float)((double)H / (2.0 * th));
  v.nearp = c.near_plane;
  v.farp = c.far_plane;
  return v;
}

LightC make_light(const mrr_gbuffer& g) {
  LightC L;
  for (int k = 0; k < 3; ++k) {
    L.ce[k] = g.cam.eye[k];
    L.cr[k] = g.cam.right[k];
    L.cu[k] = g.cam.up[k];
    L.cf[k] = g.cam.forward[k];
    L.le[k] = g.light.eye[k];
    L.lr[k] = g.light.right[k];
    L.lu[k] = g.light.up[k];
    L.lf[k] = g.light.forward[k];
  }
  L.tl = g.light.tan_half_fov;
  L.kl = (float)((double)g.shadow_size / (2.0 * (double)g.light.tan_half_fov));
  L.nearp = g.light.near_plane;
  L.farp = g.light.far_plane;
  L.S = g.shadow_size;
  return L;
}

mrr_status check_gbuffer(mrr_ctx* ctx, const mrr_gbuffer* g, bool need_device_align = true) {
  if (!g) return fail(ctx, MRR_EINVAL, "gbuffer is NULL");
  if (g->width < 1 || g->height < 1 || g->width > MAX_DIM || g->height > MAX_DIM)
    return fail(ctx, MRR_EINVAL, "frame size %dx%d outside [1, %d]", g->width, g->height, MAX_DIM);
  if (!g->depth || !g->normal) return fail(ctx, MRR_EINVAL, "depth and normal planes are required");
  if (need_device_align && !aligned(g->normal, ctx->cfg.precision == MRR_FP16 ? 8 : 16))
    return fail(ctx, MRR_EINVAL, "normal plane is not aligned to its element size");
  if (!(g->cam.tan_half_fov > 0.f) || !(g->cam.near_plane >= CAM_MIN_NEAR) || !(g->cam.far_plane > g->cam.near_plane) ||
      !(g->cam.far_plane <= CAM_MAX_FAR))
    return fail(ctx, MRR_EINVAL, "camera needs tan_half_fov > 0 and 2^-60 <= near < far <= 2^60");
  if (ctx->cfg.effect == MRR_SSGI) {
    if (!g->color) return fail(ctx, MRR_EINVAL, "SSGI needs the direct-light colour plane");
    if (need_device_align && !aligned(g->color, 8)) return fail(ctx, MRR_EINVAL, "colour plane not 8-byte aligned");
  }
  if (ctx->cfg.effect == MRR_SSM) {
    if (!g->shadow_map || g->shadow_size < 1 || g->shadow_size > MAX_DIM)
      return fail(ctx, MRR_EINVAL, "SSM needs a shadow map of side 1..%d", MAX_DIM);
    if (!(g->light.tan_half_fov > 0.f) || !(g->light.near_plane > 0.f))
      return fail(ctx, MRR_EINVAL, "light camera needs tan_half_fov > 0 and near > 0");
  }
  return MRR_OK;
}

ShadeParams make_shade_params(const mrr_ctx* ctx, const mrr_gbuffer& g) {
  ShadeParams p;
  const mrr_config& c = ctx->cfg;
  p.effect = c.effect;
  p.v = make_view(g.width, g.height, g.cam);
  if (c.effect == MRR_SSM) p.L = make_light(g);
  else std::memset(&p.L, 0, sizeof p.L);
  p.samples = c.samples;
  p.radius = c.radius;
  p.ao_bias = c.ao_bias;
  p.gi_min_dist2 = c.gi_min_dist2;
  p.light_half = c.light_size * 0.5f;
  p.shadow_bias = c.shadow_bias;
  p.nb = c.blocker_samples;
  p.np = c.pcf_samples;
  std::memcpy(p.kernel, ctx->kernel, sizeof p.kernel);
  for (int j = 0; j < MRR_MAX_SAMPLES; ++j) {
    p.kx[j] = ctx->kernel[j].x;
    p.ky[j] = ctx->kernel[j].y;
    p.kz[j] = ctx->kernel[j].z;
  }
  std::memcpy(p.btaps, ctx->btaps, sizeof p.btaps);
  std::memcpy(p.ptaps, ctx->ptaps, sizeof p.ptaps);
  return p;
}

FrameIn make_frame_in(const mrr_gbuffer& g);

// The shading parameters of level `level`: for sample-count levels above 0 (Sec. 6) every
// sample table keeps its entries 0, 2^level, 2 * 2^level, ... (ceil(n / 2^level) of n).
ShadeParams level_shade_params(const mrr_ctx* ctx, const mrr_gbuffer& g, int level) {
  ShadeParams p = make_shade_params(ctx, g);
  if (!ctx->cfg.sample_levels || level == 0) return p;
  const int step = 1 << level;
  auto thin = [&](int n) { return (n + step - 1) / step; };
  p.samples = thin(ctx->cfg.samples);
  for (int j = 0; j < MRR_MAX_SAMPLES; ++j) {
    const float4 k = j < p.samples ? ctx->kernel[j * step] : make_float4(0.f, 0.f, 0.f, 0.f);
    p.kernel[j] = k;
    p.kx[j] = k.x;
    p.ky[j] = k.y;
    p.kz[j] = k.z;
  }
  p.nb = thin(ctx->cfg.blocker_samples);
  p.np = thin(ctx->cfg.pcf_samples);
  for (int j = 0; j < MRR_MAX_TAPS; ++j) {
    p.btaps[j] = j < p.nb ? ctx->btaps[j * step] : make_float2(0.f, 0.f);
    p.ptaps[j] = j < p.np ? ctx->ptaps[j * step] : make_float2(0.f, 0.f);
  }
  return p;
}

bool fits_pools(const mrr_ctx* ctx, int W, int H);

// Pyramid gathers: build the point-sampled depth of the enabled levels above 0 (those in
// `mask`) into the context's pools and point the shading slots at them.
mrr_status pyramid_impl(mrr_ctx* ctx, const mrr_gbuffer& g, const mrr_levels* lv, unsigned mask, ShadeLevels& sl,
                        cudaStream_t s) {
  if (!ctx->cfg.pyramid_gathers) return MRR_OK;
  if (!fits_pools(ctx, g.width, g.height))
    return fail(ctx, MRR_EINVAL, "pyramid gathers: frame %dx%d exceeds the context's max size", g.width, g.height);
  PyramidParams pp;
  std::memset(&pp, 0, sizeof pp);
  pp.W = g.width;
  pp.H = g.height;
  pp.depth = g.depth;
  for (int i = 1; i < ctx->cfg.num_levels; ++i) {
    if (!ctx->cfg.enabled[i] || !((mask >> i) & 1u)) continue;
    const int k = pp.nlev++;
    pp.level[k] = i;
    pp.Wi[k] = lv->width[i];
    pp.Hi[k] = lv->height[i];
    pp.out[k] = ctx->pyr[i];
  }
  MRR_CUDA(ctx, launch_pyramid(pp, s));
  sl.pyramid = 1;
  for (int k = 0; k < sl.nlev; ++k) sl.pyr[k] = sl.level[k] > 0 ? ctx->pyr[sl.level[k]] : nullptr;
  return MRR_OK;
}

// Sample-count level `level` of frame g into c ([H][W]).
mrr_status shade_blocks_impl(mrr_ctx* ctx, const mrr_gbuffer& g, const mrr_levels* lv, int level, void* c,
                             cudaStream_t s) {
  BlockLevel b;
  b.level = level;
  b.Wi = lv->width[level];
  b.Hi = lv->height[level];
  b.list = lv->worklist[level];
  b.count = lv->counts + level;
  b.c = c;
  MRR_CUDA(ctx, launch_shade_blocks(level_shade_params(ctx, g, level), make_frame_in(g), ctx->cfg.precision, b,
                                    ctx->shade_grid, s));
  return MRR_OK;
}

FrameIn make_frame_in(const mrr_gbuffer& g) {
  FrameIn in;
  in.depth = g.depth;
  in.normal = g.normal;
  in.color = reinterpret_cast<const half4*>(g.color);
  in.smap = g.shadow_map;
  return in;
}

mrr_status check_levels(mrr_ctx* ctx, const mrr_levels* lv, bool need_lists) {
  if (!lv) return fail(ctx, MRR_EINVAL, "levels is NULL");
  const mrr_config& c = ctx->cfg;
  if (lv->num_levels != c.num_levels)
    return fail(ctx, MRR_EINVAL, "levels->num_levels %d != context num_levels %d", lv->num_levels, c.num_levels);
  const int W = lv->width[0], H = lv->height[0];
  if (W < 1 || H < 1 || W > MAX_DIM || H > MAX_DIM) return fail(ctx, MRR_EINVAL, "bad level-0 size %dx%d", W, H);
  for (int i = 0; i < c.num_levels; ++i) {
    if (lv->width[i] != level_dim(W, i) || lv->height[i] != level_dim(H, i))
      return fail(ctx, MRR_EINVAL, "level %d is %dx%d, expected %dx%d", i, lv->width[i], lv->height[i],
                  level_dim(W, i), level_dim(H, i));
    if (c.enabled[i] && (!lv->alpha[i] || !lv->stencil[i] || (need_lists && !lv->worklist[i])))
      return fail(ctx, MRR_EINVAL, "level %d buffers missing", i);
  }
  if (!lv->counts) return fail(ctx, MRR_EINVAL, "levels->counts is NULL");
  return MRR_OK;
}

MaskParams mask_params(const mrr_ctx* ctx, const mrr_levels* lv) {
  MaskParams m;
  mask_level_params(ctx->cfg, lv, m);  // the configuration was validated by mrr_create
  m.lut0 = ctx->lut0;
  for (int i = 1; i < MRR_MAX_LEVELS; ++i) m.lut[i] = ctx->lut[i];
  return m;
}

mrr_status masks_impl(mrr_ctx* ctx, const uint8_t* E, const mrr_levels* lv, cudaStream_t s) {
  const mrr_config& c = ctx->cfg;
  const int W = lv->width[0], H = lv->height[0];
  const MaskParams m = mask_params(ctx, lv);
  MRR_CUDA(ctx, launch_masks(m, E, s));
  // work lists of every enabled level in one two-pass compaction
  CompactParams cp;
  std::memset(&cp, 0, sizeof cp);
  int nchunks = 0;
  for (int i = 0; i < c.num_levels; ++i) {
    if (!c.enabled[i]) {
      cp.zero_mask |= 1 << i;
      continue;
    }
    const int l = cp.nlev++;
    cp.level_of[l] = i;
    cp.chunk_begin[l] = nchunks;
    cp.Wi[l] = lv->width[i];
    cp.Hi[l] = lv->height[i];
    cp.stencil[l] = lv->stencil[i];
    cp.list[l] = lv->worklist[i];
    nchunks += (int)(((size_t)lv->width[i] * lv->height[i] + COMPACT_CHUNK - 1) / COMPACT_CHUNK);
  }
  for (int i = c.num_levels; i < MRR_MAX_LEVELS; ++i) cp.zero_mask |= 1 << i;
  cp.chunk_begin[cp.nlev] = nchunks;
  if ((size_t)nchunks > ctx->chunk_cap)
    return fail(ctx, MRR_EINVAL, "frame %dx%d exceeds the context's max size", W, H);
  cp.chunk_counts = ctx->chunk_counts;
  cp.counts = lv->counts;
  MRR_CUDA(ctx, launch_compact(cp, s));
  return MRR_OK;
}

mrr_status edges_impl(mrr_ctx* ctx, const mrr_gbuffer* g, uint8_t* E, cudaStream_t s, uint32_t* zero = nullptr,
                      int zero_words = 0, uint32_t* ebits = nullptr, bool concurrent = false) {
  EdgeParams p;
  std::memset(&p, 0, sizeof p);
  p.v = make_view(g->width, g->height, g->cam);
  p.ssm = ctx->cfg.effect == MRR_SSM;
  if (p.ssm) p.L = make_light(*g);
  p.depth_rel = ctx->cfg.depth_rel;
  p.normal_cos = ctx->cfg.normal_cos;
  p.shadow_bias = ctx->cfg.shadow_bias;
  p.fault = ctx->fault;
  p.zero = zero;
  p.zero_words = zero_words;
  p.ebits = ebits;
  p.ewords = (g->width + 31) / 32;
  if (p.ssm && ctx->sbits && g->width <= ctx->pool_W && g->height <= ctx->pool_H) p.sbits = ctx->sbits;
  p.concurrent = concurrent ? 1 : 0;
  const int h = ctx->cfg.precision == MRR_FP16;
  MRR_CUDA(ctx, launch_edges(p, g->depth, g->normal, h, (const float*)g->shadow_map, E, s));
  return MRR_OK;
}

mrr_levels pool_levels(mrr_ctx* ctx, int W, int H) {
  mrr_levels lv;
  std::memset(&lv, 0, sizeof lv);
  lv.num_levels = ctx->cfg.num_levels;
  for (int i = 0; i < ctx->cfg.num_levels; ++i) {
    lv.width[i] = level_dim(W, i);
    lv.height[i] = level_dim(H, i);
    lv.alpha[i] = ctx->alpha[i];
    lv.stencil[i] = ctx->stencil[i];
    lv.worklist[i] = ctx->worklist[i];
  }
  lv.counts = ctx->counts;
  lv.label = nullptr;
  return lv;
}

// The step-wise blending of Sec. 3.3: one chain launch per finer enabled level (and a
// last one at level 0), intermediate composites in the context's pools.  With
// compact_level0, level 0's blend is left to the caller (level 0's list).
mrr_status chain_impl(mrr_ctx* ctx, const mrr_levels* lv, void* const* c, float* out, cudaStream_t s,
                      bool compact_level0) {
  const mrr_config& cf = ctx->cfg;
  int j = cf.num_levels - 1;
  const void* src = c[j];
  bool src_sub = true;
  for (int i = cf.num_levels - 2; i >= 0; --i) {
    if (i > 0 && !cf.enabled[i]) continue;
    ChainParams cp;
    std::memset(&cp, 0, sizeof cp);
    cp.C = channels(cf);
    cp.half_store = cf.precision == MRR_FP16;
    cp.i = i;
    cp.j = j;
    cp.Wi = lv->width[i];
    cp.Hi = lv->height[i];
    cp.Wj = lv->width[j];
    cp.Hj = lv->height[j];
    cp.weight = cf.weight[i];
    cp.blend = cf.enabled[i] && !(i == 0 && compact_level0);
    cp.alpha = lv->alpha[i];
    cp.stencil = lv->stencil[i];
    cp.c = c[i];
    cp.src = src;
    cp.src_sub = src_sub;
    cp.dst = i == 0 ? out : ctx->comp[i];
    MRR_CUDA(ctx, launch_chain(cp, s));
    src = cp.dst;
    src_sub = false;
    j = i;
  }
  return MRR_OK;
}

mrr_status merge_impl(mrr_ctx* ctx, const mrr_levels* lv, void* const* c, float* out, cudaStream_t s,
                      bool compact_level0 = false, const float* depth = nullptr) {
  const mrr_config& cf = ctx->cfg;
  if (cf.disjoint) {
    MergeParams mp;
    std::memset(&mp, 0, sizeof mp);
    mp.W = lv->width[0];
    mp.H = lv->height[0];
    mp.L = cf.num_levels;
    mp.C = channels(cf);
    mp.half_store = cf.precision == MRR_FP16;
    for (int i = 0; i < cf.num_levels; ++i) {
      mp.enabled[i] = cf.enabled[i];
      mp.Wi[i] = lv->width[i];
      mp.Hi[i] = lv->height[i];
      mp.stencil[i] = lv->stencil[i];
      mp.c[i] = c[i];
    }
    MRR_CUDA(ctx, launch_merge_disjoint(mp, out, s));
    return MRR_OK;
  }
  if (cf.merge_mode == 2 && !cf.sample_levels) {
    if (!depth) return fail(ctx, MRR_EINVAL, "the bilateral merge needs the frame's depth");
    MergeParams mp;
    std::memset(&mp, 0, sizeof mp);
    mp.W = lv->width[0];
    mp.H = lv->height[0];
    mp.L = cf.num_levels;
    mp.C = channels(cf);
    mp.half_store = cf.precision == MRR_FP16;
    for (int i = 0; i < cf.num_levels; ++i) {
      mp.enabled[i] = cf.enabled[i];
      mp.Wi[i] = lv->width[i];
      mp.Hi[i] = lv->height[i];
      mp.weight[i] = cf.weight[i];
      mp.alpha[i] = lv->alpha[i];
      mp.stencil[i] = lv->stencil[i];
      mp.c[i] = c[i];
    }
    if (compact_level0) mp.enabled[0] = 0;  // blended afterwards from level 0's list
    MRR_CUDA(ctx, launch_merge_bilateral(mp, depth, cf.blur_depth_rel, out, s));
  } else if (cf.merge_mode == 1 && cf.num_levels > 1) {
    mrr_status st = chain_impl(ctx, lv, c, out, s, compact_level0);
    if (st != MRR_OK) return st;
  } else if (cf.sample_levels && cf.num_levels > 1) {
    MergeParams mp;
    std::memset(&mp, 0, sizeof mp);
    mp.W = lv->width[0];
    mp.H = lv->height[0];
    mp.L = cf.num_levels;
    mp.C = channels(cf);
    mp.half_store = cf.precision == MRR_FP16;
    for (int i = 0; i < cf.num_levels; ++i) {
      mp.enabled[i] = cf.enabled[i];
      mp.Wi[i] = lv->width[i];
      mp.Hi[i] = lv->height[i];
      mp.weight[i] = cf.weight[i];
      mp.alpha[i] = lv->alpha[i];
      mp.stencil[i] = lv->stencil[i];
      mp.c[i] = c[i];
    }
    if (compact_level0) mp.enabled[0] = 0;  // blended afterwards from level 0's list
    MRR_CUDA(ctx, launch_merge_samples(mp, out, s));
  } else {
    MergeParams mp;
    std::memset(&mp, 0, sizeof mp);
    mp.W = lv->width[0];
    mp.H = lv->height[0];
    mp.L = cf.num_levels;
    mp.C = channels(cf);
    mp.half_store = cf.precision == MRR_FP16;
    for (int i = 0; i < cf.num_levels; ++i) {
      mp.enabled[i] = cf.enabled[i];
      mp.Wi[i] = lv->width[i];
      mp.Hi[i] = lv->height[i];
      mp.weight[i] = cf.weight[i];
      mp.alpha[i] = lv->alpha[i];
      mp.stencil[i] = lv->stencil[i];
      mp.c[i] = c[i];
    }
    if (compact_level0) mp.enabled[0] = 0;  // blended afterwards from level 0's list
    MRR_CUDA(ctx, launch_merge(mp, out, s));
  }
  if (compact_level0 && cf.enabled[0]) {
    Blend0Params bp;
    std::memset(&bp, 0, sizeof bp);
    bp.W = lv->width[0];
    bp.H = lv->height[0];
    bp.C = channels(cf);
    bp.half_store = cf.precision == MRR_FP16;
    bp.weight = cf.weight[0];
    bp.list = ctx->worklist[0];
    bp.count = ctx->counts;
    bp.a0c = ctx->alpha[0];
    bp.c0c = ctx->cbuf[0];
    MRR_CUDA(ctx, launch_blend0(bp, out, s));
  }
  return MRR_OK;
}

// Blur parameters for frame g with levels lv; slots are added by the caller.
BlurParams blur_params(const mrr_ctx* ctx, const mrr_gbuffer* g, const mrr_levels* lv) {
  BlurParams bp;
  std::memset(&bp, 0, sizeof bp);
  bp.W = g->width;
  bp.H = g->height;
  bp.C = channels(ctx->cfg);
  bp.half_store = ctx->cfg.precision == MRR_FP16;
  bp.rel = ctx->cfg.blur_depth_rel;
  bp.depth = g->depth;
  return bp;
}

void add_blur_slot(BlurParams& bp, const mrr_levels* lv, int level, const void* c, void* b) {
  const int k = bp.nlev++;
  bp.level[k] = level;
  bp.Wi[k] = lv->width[level];
  bp.Hi[k] = lv->height[level];
  bp.tile_begin[k + 1] = bp.tile_begin[k] + blur_tiles(bp.Wi[k], bp.Hi[k]);
  bp.stencil[k] = lv->stencil[level];
  bp.c[k] = c;
  bp.b[k] = b;
}

// Sec. 4.1: blur the pool sub-images of the levels cfg.blur names (one launch); c_merge[i]
// receives the sub-image the blend reads for level i (blurred or not).
mrr_status blur_pools(mrr_ctx* ctx, const mrr_gbuffer* g, const mrr_levels* lv, void** c_merge, cudaStream_t s) {
  BlurParams bp = blur_params(ctx, g, lv);
  for (int i = 0; i < MRR_MAX_LEVELS; ++i) c_merge[i] = ctx->cbuf[i];
  for (int i = 1; i < ctx->cfg.num_levels; ++i) {
    if (!ctx->cfg.blur[i]) continue;
    add_blur_slot(bp, lv, i, ctx->cbuf[i], ctx->bbuf[i]);
    c_merge[i] = ctx->bbuf[i];
  }
  if (bp.nlev) MRR_CUDA(ctx, launch_blur(bp, s));
  return MRR_OK;
}

mrr_status render_launches(mrr_ctx* ctx, const mrr_gbuffer* g, float* out, cudaStream_t s);

// mrr_render's launches depend only on the frame descriptor (pointers, sizes, cameras)
// and the output pointer: the first call with a new descriptor captures them into a
// graph on an internal stream, later calls with the same descriptor replay it on the
// caller's stream (one launch instead of six).
mrr_gbuffer canonical_key(const mrr_gbuffer* g) {  // field copy: padding bytes are zero
  mrr_gbuffer k;
  std::memset(&k, 0, sizeof k);
  k.width = g->width;
  k.height = g->height;
  k.depth = g->depth;
  k.normal = g->normal;
  k.color = g->color;
  k.shadow_map = g->shadow_map;
  k.shadow_size = g->shadow_size;
  k.cam = g->cam;
  k.light = g->light;
  return k;
}

mrr_status render_impl(mrr_ctx* ctx, const mrr_gbuffer* g, float* out, cudaStream_t s) {
  if (!ctx->use_graph || ctx->trace_begin) return render_launches(ctx, g, out, s);
  const mrr_gbuffer key = canonical_key(g);
  int hit = -1;
  for (int e = 0; e < 2; ++e)
    if (ctx->graph_exec[e] && out == ctx->graph_out[e] && std::memcmp(&ctx->graph_key[e], &key, sizeof key) == 0)
      hit = e;
  if (hit < 0) {
    hit = ctx->graph_next;
    ctx->graph_next ^= 1;
    if (ctx->graph_exec[hit]) {
      cudaGraphExecDestroy(ctx->graph_exec[hit]);
      ctx->graph_exec[hit] = nullptr;
    }
    if (!ctx->capture_stream) MRR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    MRR_CUDA(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    const uint64_t before = launch_counter().load();
    mrr_status st = render_launches(ctx, g, out, ctx->capture_stream);
    // captured launches do not run: count them per replay instead
    ctx->graph_kernels[hit] = launch_counter().load() - before;
    launch_counter().fetch_sub(ctx->graph_kernels[hit]);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (st != MRR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(ctx, MRR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph_exec[hit], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->graph_exec[hit] = nullptr;
      return fail(ctx, MRR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    ctx->graph_key[hit] = key;
    ctx->graph_out[hit] = out;
  }
  MRR_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec[hit], s));
  count_launches((int)ctx->graph_kernels[hit]);
  ++ctx->graph_replays;
  return MRR_OK;
}

// A frame fits the context's pools (level buffers and work lists).
bool fits_pools(const mrr_ctx* ctx, int W, int H) {
  for (int i = 0; i < ctx->cfg.num_levels; ++i)
    if ((size_t)level_dim(W, i) * level_dim(H, i) > (size_t)level_dim(ctx->pool_W, i) * level_dim(ctx->pool_H, i))
      return false;
  return true;
}

mrr_status render_launches_staged(mrr_ctx* ctx, const mrr_gbuffer* g, float* out, cudaStream_t s);

// The frame path's first two launches (at least two levels): edges, bit-packed, also
// clearing the per-level counts; masks that also write every enabled level's work list
// and level 0's a_0 list-aligned (into the level-0 alpha pool).
mrr_status frame_masks(mrr_ctx* ctx, const mrr_gbuffer* g, mrr_levels* lv, cudaStream_t s, bool batched = false) {
  const mrr_config& c = ctx->cfg;
  const int W = g->width, H = g->height;
  mrr_status st = edges_impl(ctx, g, ctx->edges, s, ctx->counts, MRR_MAX_LEVELS, ctx->ebits, batched);
  if (st != MRR_OK) return st;
  *lv = pool_levels(ctx, W, H);
  MaskParams m = mask_params(ctx, lv);
  m.label = nullptr;
  m.a0c = ctx->alpha[0];
  m.ebits = ctx->ebits;
  m.ewords = (W + 31) / 32;
  for (int i = 0; i < c.num_levels; ++i) m.list[i] = c.enabled[i] ? ctx->worklist[i] : nullptr;
  m.counts = ctx->counts;
  MRR_CUDA(ctx, launch_masks(m, ctx->edges, s));
  return MRR_OK;
}

// With at least two levels: edges (also clearing the per-level counts; the edge image
// bit-packed), masks that also write the work lists and level 0's a_0 list-aligned, one
// shading launch over every level (level 0's c_0 list-aligned too), the blur of the
// levels cfg.blur names (if any), the merge of the levels above 0, and level 0 blended
// in over its list.  Level 0's full-resolution a_0,
// S_0 and c_0 never reach memory, and no compaction launch is needed.
mrr_status render_launches(mrr_ctx* ctx, const mrr_gbuffer* g, float* out, cudaStream_t s) {
  const mrr_config& c = ctx->cfg;
  const int W = g->width, H = g->height;
  if (c.num_levels < 2 || c.disjoint) return render_launches_staged(ctx, g, out, s);
  if (!fits_pools(ctx, W, H)) return fail(ctx, MRR_EINVAL, "frame %dx%d exceeds the context's max size", W, H);
  mrr_levels lv;
  mrr_status st = frame_masks(ctx, g, &lv, s);
  if (st != MRR_OK) return st;
  ShadeParams p = make_shade_params(ctx, *g);
  ShadeLevels sl;
  std::memset(&sl, 0, sizeof sl);
  for (int i = 0; i < c.num_levels; ++i) {
    if (!c.enabled[i] || (c.sample_levels && i > 0)) continue;
    const int k = sl.nlev++;
    sl.level[k] = i;
    sl.list[k] = ctx->worklist[i];
    sl.c[k] = ctx->cbuf[i];
    sl.Wi[k] = lv.width[i];
    sl.Hi[k] = lv.height[i];
    if (i == 0) sl.compact |= 1 << k;
  }
  sl.counts = ctx->counts;
  st = pyramid_impl(ctx, *g, &lv, ~0u, sl, s);
  if (st != MRR_OK) return st;
  if (ctx->trace_begin) MRR_CUDA(ctx, cudaEventRecord(ctx->trace_begin, s));
  if (sl.nlev)
    MRR_CUDA(ctx, launch_shade_levels(p, make_frame_in(*g), c.precision, sl, ctx->shade_grid, ctx->split_texel, s));
  if (ctx->trace_end) MRR_CUDA(ctx, cudaEventRecord(ctx->trace_end, s));
  if (c.sample_levels)
    for (int i = 1; i < c.num_levels; ++i) {
      if (!c.enabled[i]) continue;
      st = shade_blocks_impl(ctx, *g, &lv, i, ctx->cbuf[i], s);
      if (st != MRR_OK) return st;
    }
  void* cm[MRR_MAX_LEVELS];
  st = blur_pools(ctx, g, &lv, cm, s);
  if (st != MRR_OK) return st;
  return merge_impl(ctx, &lv, cm, out, s, true, g->depth);
}

// One level only (level 0 is the coarsest), or the disjoint-tile ablation: edges, masks,
// compaction, shading, merge.
mrr_status render_launches_staged(mrr_ctx* ctx, const mrr_gbuffer* g, float* out, cudaStream_t s) {
  const int W = g->width, H = g->height;
  mrr_status st = edges_impl(ctx, g, ctx->edges, s);
  if (st != MRR_OK) return st;
  mrr_levels lv = pool_levels(ctx, W, H);
  st = masks_impl(ctx, ctx->edges, &lv, s);
  if (st != MRR_OK) return st;
  ShadeParams p = make_shade_params(ctx, *g);
  ShadeLevels sl;
  std::memset(&sl, 0, sizeof sl);
  for (int i = 0; i < ctx->cfg.num_levels; ++i) {
    if (!ctx->cfg.enabled[i]) continue;
    const int k = sl.nlev++;
    sl.level[k] = i;
    sl.list[k] = ctx->worklist[i];
    sl.c[k] = ctx->cbuf[i];
    sl.Wi[k] = lv.width[i];
    sl.Hi[k] = lv.height[i];
  }
  sl.counts = ctx->counts;
  MRR_CUDA(ctx, launch_shade_levels(p, make_frame_in(*g), ctx->cfg.precision, sl, ctx->shade_grid,
                                    ctx->split_texel, s));
  return merge_impl(ctx, &lv, ctx->cbuf, out, s, false, g->depth);
}

void free_pools(mrr_ctx* ctx) {
  for (int e = 0; e < 2; ++e) {
    if (ctx->graph_exec[e]) cudaGraphExecDestroy(ctx->graph_exec[e]);
    ctx->graph_exec[e] = nullptr;
  }
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  ctx->capture_stream = nullptr;
  for (auto& hs : ctx->hset) {
    cudaFree(hs.depth);
    cudaFree(hs.normal);
    cudaFree(hs.color);
    cudaFree(hs.smap);
    cudaFree(hs.out);
    if (hs.loaded) cudaEventDestroy(hs.loaded);
    if (hs.rendered) cudaEventDestroy(hs.rendered);
    if (hs.done) cudaEventDestroy(hs.done);
    hs = mrr_ctx::HostSet();
  }
  for (cudaStream_t* st : {&ctx->s_in, &ctx->s_comp, &ctx->s_out}) {
    if (*st) cudaStreamDestroy(*st);
    *st = nullptr;
  }
  cudaFree(ctx->edges);
  cudaFree(ctx->ebits);
  cudaFree(ctx->sbits);
  for (int i = 0; i < MRR_MAX_LEVELS; ++i) {
    cudaFree(ctx->alpha[i]);
    cudaFree(ctx->stencil[i]);
    cudaFree(ctx->worklist[i]);
    cudaFree(ctx->cbuf[i]);
    cudaFree(ctx->bbuf[i]);
    cudaFree(ctx->comp[i]);
    cudaFree(ctx->pyr[i]);
  }
  cudaFree(ctx->counts);
  cudaFree(ctx->chunk_counts);
  cudaFree(ctx->lut0);
  for (float*& t : ctx->lut) {
    cudaFree(t);
    t = nullptr;
  }
  cudaFree(ctx->fault);
  cudaFree(ctx->h_depth);
  cudaFree(ctx->h_normal);
  cudaFree(ctx->h_color);
  cudaFree(ctx->h_smap);
  cudaFree(ctx->h_out);
}

mrr_status alloc_pools(mrr_ctx* ctx) {
  const mrr_config& c = ctx->cfg;
  const int W = c.max_width, H = c.max_height;
  ctx->pool_W = W;
  ctx->pool_H = H;
  const size_t npx = (size_t)W * H;
  MRR_CUDA(ctx, cudaMalloc(&ctx->edges, npx));
  MRR_CUDA(ctx, cudaMalloc(&ctx->ebits, (size_t)((W + 31) / 32) * H * sizeof(uint32_t)));
  if (c.effect == MRR_SSM) MRR_CUDA(ctx, cudaMalloc(&ctx->sbits, (size_t)((W + 31) / 32) * H * sizeof(uint32_t)));
  size_t chunks = 0;
  for (int i = 0; i < c.num_levels; ++i) {
    const size_t n = (size_t)level_dim(W, i) * level_dim(H, i);
    MRR_CUDA(ctx, cudaMalloc(&ctx->alpha[i], n * sizeof(float)));
    MRR_CUDA(ctx, cudaMalloc(&ctx->stencil[i], n));
    if (c.enabled[i]) {
      MRR_CUDA(ctx, cudaMalloc(&ctx->worklist[i], n * sizeof(uint32_t)));
      // sample-count levels keep every level's sub-image at full resolution
      MRR_CUDA(ctx, cudaMalloc(&ctx->cbuf[i], (c.sample_levels && i > 0 ? npx : n) * cbytes(c)));
    }
    if (c.blur[i]) MRR_CUDA(ctx, cudaMalloc(&ctx->bbuf[i], n * cbytes(c)));
    if (c.merge_mode == 1 && i >= 1 && i < c.num_levels - 1 && c.enabled[i])
      MRR_CUDA(ctx, cudaMalloc(&ctx->comp[i], n * (c.effect == MRR_SSGI ? 16 : 4)));
    if (c.pyramid_gathers && i >= 1 && c.enabled[i]) MRR_CUDA(ctx, cudaMalloc(&ctx->pyr[i], n * sizeof(float)));
    chunks += (n + COMPACT_CHUNK - 1) / COMPACT_CHUNK;
  }
  // level 0's horizontal blur for every (2R+1)-bit window, summed exactly as the
  // definition sums it: ascending taps, s = s + g[t] for every set tap, in float
  if (c.enabled[0] && c.num_levels > 1 && !c.force_level0 && ctx->R[0] > 0 && (1 << (2 * ctx->R[0] + 1)) <= MASK_LUT_MAX) {
    const int n = 1 << (2 * ctx->R[0] + 1);
    float host[MASK_LUT_MAX];
    for (int b = 0; b < n; ++b) {
      float acc = 0.0f;
      for (int t = 0; t <= 2 * ctx->R[0]; ++t)
        if ((b >> t) & 1) acc = acc + ctx->gauss[0][t];
      host[b] = acc;
    }
    MRR_CUDA(ctx, cudaMalloc(&ctx->lut0, n * sizeof(float)));
    MRR_CUDA(ctx, cudaMemcpy(ctx->lut0, host, n * sizeof(float), cudaMemcpyHostToDevice));
  }
  // the same tables for the blurred levels above 0, summed the same way
  for (int i = 1; i < c.num_levels; ++i) {
    const int R = ctx->R[i];
    if (R <= 0 || R > MASK_LUT_GLOBAL_R) continue;
    const int n = 1 << (2 * R + 1);
    std::vector<float> host(n);
    for (int b = 0; b < n; ++b) {
      float acc = 0.0f;
      for (int t = 0; t <= 2 * R; ++t)
        if ((b >> t) & 1) acc = acc + ctx->gauss[i][t];
      host[b] = acc;
    }
    MRR_CUDA(ctx, cudaMalloc(&ctx->lut[i], n * sizeof(float)));
    MRR_CUDA(ctx, cudaMemcpy(ctx->lut[i], host.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  }
  MRR_CUDA(ctx, cudaMalloc(&ctx->counts, MRR_MAX_LEVELS * sizeof(uint32_t)));
  MRR_CUDA(ctx, cudaMemset(ctx->counts, 0, MRR_MAX_LEVELS * sizeof(uint32_t)));
  MRR_CUDA(ctx, cudaMalloc(&ctx->fault, sizeof(uint32_t)));
  MRR_CUDA(ctx, cudaMemset(ctx->fault, 0, sizeof(uint32_t)));
  ctx->chunk_cap = chunks;
  MRR_CUDA(ctx, cudaMalloc(&ctx->chunk_counts, chunks * sizeof(uint32_t)));
  return MRR_OK;
}

}  // namespace

extern "C" {

mrr_status mrr_level_dims(int width, int height, int level, int* level_width, int* level_height) {
  if (width < 1 || height < 1 || width > MAX_DIM || height > MAX_DIM || level < 0 || level >= MRR_MAX_LEVELS ||
      !level_width || !level_height)
    return MRR_EINVAL;
  *level_width = level_dim(width, level);
  *level_height = level_dim(height, level);
  return MRR_OK;
}

mrr_status mrr_create(const mrr_config* cfg, mrr_ctx** out) {
  if (!out) return MRR_EINVAL;
  *out = nullptr;
  if (!cfg) return MRR_EINVAL;
  const mrr_config& c = *cfg;
  if (c.effect < MRR_SSAO || c.effect > MRR_SSGI) return MRR_EINVAL;
  if (c.precision != MRR_FP32 && c.precision != MRR_FP16) return MRR_EINVAL;
  if (c.num_levels < 1 || c.num_levels > MRR_MAX_LEVELS || !c.enabled[c.num_levels - 1]) return MRR_EINVAL;
  for (int i = 0; i < c.num_levels; ++i) {
    if (!c.enabled[i]) continue;
    if (i < c.num_levels - 1 && !(i == 0 && c.force_level0)) {
      if (!(c.sigma2[i] > 0.f) || std::ceil(3.0 * std::sqrt((double)c.sigma2[i])) > 6.0) return MRR_EINVAL;
    }
    if (!(c.weight[i] >= 0.f)) return MRR_EINVAL;
  }
  if (c.max_width < 1 || c.max_height < 1 || c.max_width > MAX_DIM || c.max_height > MAX_DIM) return MRR_EINVAL;
  for (int i = 0; i < MRR_MAX_LEVELS; ++i) {
    if (c.blur[i] != 0 && c.blur[i] != 1) return MRR_EINVAL;
    if (c.blur[i] && (i == 0 || i >= c.num_levels || !c.enabled[i])) return MRR_EINVAL;
  }
  if (!(c.blur_depth_rel >= 0.f) || !(c.blur_depth_rel <= FLT_MAX)) return MRR_EINVAL;
  if (c.merge_mode < 0 || c.merge_mode > 2) return MRR_EINVAL;
  if (c.sample_levels != 0 && c.sample_levels != 1) return MRR_EINVAL;
  if (c.pyramid_gathers != 0 && c.pyramid_gathers != 1) return MRR_EINVAL;
  if (c.pyramid_gathers && (c.effect != MRR_SSAO || c.sample_levels)) return MRR_EINVAL;
  if (c.disjoint != 0 && c.disjoint != 1) return MRR_EINVAL;
  if (c.disjoint) {  // the ablation stands alone: no blur, step-wise or bilateral merge, sample levels, pyramid
    if (c.merge_mode != 0 || c.sample_levels || c.pyramid_gathers) return MRR_EINVAL;
    for (int i = 0; i < MRR_MAX_LEVELS; ++i)
      if (c.blur[i]) return MRR_EINVAL;
  }
  if (c.sample_levels) {  // full-resolution sub-images: no level blur, direct blend only
    if (c.merge_mode != 0) return MRR_EINVAL;
    for (int i = 0; i < MRR_MAX_LEVELS; ++i)
      if (c.blur[i]) return MRR_EINVAL;
  }
  for (int v : {c.lanes_per_texel, c.lanes_per_pixel})
    if (v != 0 && v != 1 && v != 2 && v != 4) return MRR_EINVAL;
  if (c.effect != MRR_SSM) {
    if (c.samples < 1 || c.samples > MRR_MAX_SAMPLES || !c.kernel || !(c.radius > 0.f)) return MRR_EINVAL;
  } else {
    if (c.blocker_samples < 1 || c.blocker_samples > MRR_MAX_TAPS || c.pcf_samples < 1 ||
        c.pcf_samples > MRR_MAX_TAPS || !c.blocker_taps || !c.pcf_taps || !(c.light_size > 0.f))
      return MRR_EINVAL;
  }
  mrr_ctx* ctx = new (std::nothrow) mrr_ctx();
  if (!ctx) return MRR_ENOMEM;
  ctx->cfg = c;
  ctx->cfg.kernel = ctx->cfg.blocker_taps = ctx->cfg.pcf_taps = nullptr;
  std::memset(ctx->kernel, 0, sizeof ctx->kernel);
  std::memset(ctx->btaps, 0, sizeof ctx->btaps);
  std::memset(ctx->ptaps, 0, sizeof ctx->ptaps);
  if (c.kernel)
    for (int j = 0; j < c.samples; ++j)
      ctx->kernel[j] = make_float4(c.kernel[4 * j], c.kernel[4 * j + 1], c.kernel[4 * j + 2], c.kernel[4 * j + 3]);
  if (c.effect == MRR_SSM) {
    for (int j = 0; j < c.blocker_samples; ++j) ctx->btaps[j] = make_float2(c.blocker_taps[2 * j], c.blocker_taps[2 * j + 1]);
    for (int j = 0; j < c.pcf_samples; ++j) ctx->ptaps[j] = make_float2(c.pcf_taps[2 * j], c.pcf_taps[2 * j + 1]);
  }
  std::memset(ctx->gauss, 0, sizeof ctx->gauss);
  for (int i = 0; i < c.num_levels; ++i) {
    ctx->R[i] = 0;
    if (c.enabled[i] && i < c.num_levels - 1 && c.sigma2[i] > 0.f) ctx->R[i] = mask_gauss((double)c.sigma2[i], ctx->gauss[i]);
  }
  mrr_status st = alloc_pools(ctx);
  if (st != MRR_OK) {
    free_pools(ctx);
    delete ctx;
    return st == MRR_ECUDA ? MRR_ENOMEM : st;
  }
  ctx->shade_grid = shade_grid_blocks();
  edges_prepare();
  if (c.lanes_per_texel) ctx->split_texel = c.lanes_per_texel;
  if (c.lanes_per_pixel) ctx->split_pixel = c.lanes_per_pixel;
  ctx->use_graph = c.no_graph == 0;
  *out = ctx;
  return MRR_OK;
}

void mrr_destroy(mrr_ctx* ctx) {
  if (!ctx) return;
  free_pools(ctx);
  delete ctx;
}

const char* mrr_last_error(mrr_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

mrr_status mrr_check_reciprocal(uint32_t first_bits, uint32_t last_bits, uint64_t* mismatches) {
  if (!mismatches || last_bits < first_bits) return MRR_EINVAL;
  unsigned long long* bad = nullptr;
  if (cudaMalloc(&bad, sizeof *bad) != cudaSuccess) return MRR_ENOMEM;
  unsigned long long host = 0;
  bool ok = cudaMemset(bad, 0, sizeof *bad) == cudaSuccess &&
            launch_check_reciprocal(first_bits, last_bits, bad, nullptr) == cudaSuccess &&
            cudaMemcpy(&host, bad, sizeof host, cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(bad);
  if (!ok) return MRR_ECUDA;
  *mismatches = host;
  return MRR_OK;
}

mrr_status mrr_fault_flags(mrr_ctx* ctx, uint32_t* flags, int clear) {
  if (!ctx || !flags) return MRR_EINVAL;
  MRR_CUDA(ctx, cudaDeviceSynchronize());
  MRR_CUDA(ctx, cudaMemcpy(flags, ctx->fault, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (clear) MRR_CUDA(ctx, cudaMemset(ctx->fault, 0, sizeof(uint32_t)));
  return MRR_OK;
}

mrr_status mrr_check_wait_timeout(mrr_ctx* ctx, uint32_t* flags) {
  if (!ctx || !flags) return MRR_EINVAL;
  MRR_CUDA(ctx, cudaDeviceSynchronize());
  MRR_CUDA(ctx, launch_check_wait(ctx->fault, nullptr));
  MRR_CUDA(ctx, cudaDeviceSynchronize());
  MRR_CUDA(ctx, cudaMemcpy(flags, ctx->fault, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return MRR_OK;
}

mrr_status mrr_edges(mrr_ctx* ctx, const mrr_gbuffer* g, uint8_t* edges_dev, void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  if (!edges_dev) return fail(ctx, MRR_EINVAL, "edges_dev is NULL");
  return edges_impl(ctx, g, edges_dev, (cudaStream_t)stream);
}

mrr_status mrr_masks(mrr_ctx* ctx, const uint8_t* edges_dev, const mrr_levels* lv, void* stream) {
  if (!ctx) return MRR_EINVAL;
  if (!edges_dev) return fail(ctx, MRR_EINVAL, "edges_dev is NULL");
  mrr_status st = check_levels(ctx, lv, true);
  if (st != MRR_OK) return st;
  if (lv->width[0] > ctx->pool_W || lv->height[0] > ctx->pool_H) {
    // the chunk-count scratch is sized by texel count; allow any shape that fits it
    size_t need = 0;
    for (int i = 0; i < ctx->cfg.num_levels; ++i)
      if (ctx->cfg.enabled[i]) need += ((size_t)lv->width[i] * lv->height[i] + COMPACT_CHUNK - 1) / COMPACT_CHUNK;
    if (need > ctx->chunk_cap) return fail(ctx, MRR_EINVAL, "frame exceeds the context's max size");
  }
  return masks_impl(ctx, edges_dev, lv, (cudaStream_t)stream);
}

mrr_status mrr_shade_level(mrr_ctx* ctx, int level, const mrr_gbuffer* g, const mrr_levels* lv, void* c_level_dev,
                           void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  st = check_levels(ctx, lv, true);
  if (st != MRR_OK) return st;
  if (level < 0 || level >= ctx->cfg.num_levels || !ctx->cfg.enabled[level])
    return fail(ctx, MRR_EINVAL, "level %d is not an enabled level", level);
  if (lv->width[0] != g->width || lv->height[0] != g->height)
    return fail(ctx, MRR_EINVAL, "levels are for %dx%d, frame is %dx%d", lv->width[0], lv->height[0], g->width,
                g->height);
  if (!c_level_dev || !aligned(c_level_dev, cbytes(ctx->cfg)))
    return fail(ctx, MRR_EINVAL, "c_level_dev is NULL or misaligned");
  if (ctx->cfg.sample_levels && level > 0) return shade_blocks_impl(ctx, *g, lv, level, c_level_dev, (cudaStream_t)stream);
  ShadeParams p = make_shade_params(ctx, *g);
  ShadeLevels sl;
  std::memset(&sl, 0, sizeof sl);
  sl.nlev = 1;
  sl.level[0] = level;
  sl.list[0] = lv->worklist[level];
  sl.c[0] = c_level_dev;
  sl.Wi[0] = lv->width[level];
  sl.Hi[0] = lv->height[level];
  sl.counts = lv->counts;
  st = pyramid_impl(ctx, *g, lv, 1u << level, sl, (cudaStream_t)stream);
  if (st != MRR_OK) return st;
  MRR_CUDA(ctx, launch_shade_levels(p, make_frame_in(*g), ctx->cfg.precision, sl, ctx->shade_grid,
                                    ctx->split_texel, (cudaStream_t)stream));
  return MRR_OK;
}

mrr_status mrr_shade_levels(mrr_ctx* ctx, const mrr_gbuffer* g, const mrr_levels* lv, void* const* c_levels_dev,
                            void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  st = check_levels(ctx, lv, true);
  if (st != MRR_OK) return st;
  if (lv->width[0] != g->width || lv->height[0] != g->height)
    return fail(ctx, MRR_EINVAL, "levels are for %dx%d, frame is %dx%d", lv->width[0], lv->height[0], g->width,
                g->height);
  if (!c_levels_dev) return fail(ctx, MRR_EINVAL, "c_levels_dev is NULL");
  ShadeLevels sl;
  std::memset(&sl, 0, sizeof sl);
  for (int i = 0; i < ctx->cfg.num_levels; ++i) {
    if (!ctx->cfg.enabled[i]) continue;
    if (!c_levels_dev[i] || !aligned(c_levels_dev[i], cbytes(ctx->cfg)))
      return fail(ctx, MRR_EINVAL, "sub-image %d is NULL or misaligned", i);
    if (ctx->cfg.sample_levels && i > 0) continue;  // shaded below, at full resolution
    const int k = sl.nlev++;
    sl.level[k] = i;
    sl.list[k] = lv->worklist[i];
    sl.c[k] = c_levels_dev[i];
    sl.Wi[k] = lv->width[i];
    sl.Hi[k] = lv->height[i];
  }
  sl.counts = lv->counts;
  st = pyramid_impl(ctx, *g, lv, ~0u, sl, (cudaStream_t)stream);
  if (st != MRR_OK) return st;
  ShadeParams p = make_shade_params(ctx, *g);
  if (sl.nlev)
    MRR_CUDA(ctx, launch_shade_levels(p, make_frame_in(*g), ctx->cfg.precision, sl, ctx->shade_grid,
                                      ctx->split_texel, (cudaStream_t)stream));
  if (ctx->cfg.sample_levels)
    for (int i = 1; i < ctx->cfg.num_levels; ++i) {
      if (!ctx->cfg.enabled[i]) continue;
      st = shade_blocks_impl(ctx, *g, lv, i, c_levels_dev[i], (cudaStream_t)stream);
      if (st != MRR_OK) return st;
    }
  return MRR_OK;
}

mrr_status mrr_blur_level(mrr_ctx* ctx, int level, const mrr_gbuffer* g, const mrr_levels* lv,
                          const void* c_level_dev, void* b_level_dev, void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  st = check_levels(ctx, lv, false);
  if (st != MRR_OK) return st;
  if (level < 1 || level >= ctx->cfg.num_levels || !ctx->cfg.enabled[level])
    return fail(ctx, MRR_EINVAL, "level %d is not an enabled level above 0", level);
  if (lv->width[0] != g->width || lv->height[0] != g->height)
    return fail(ctx, MRR_EINVAL, "levels are for %dx%d, frame is %dx%d", lv->width[0], lv->height[0], g->width,
                g->height);
  if (!c_level_dev || !b_level_dev || !aligned(c_level_dev, cbytes(ctx->cfg)) ||
      !aligned(b_level_dev, cbytes(ctx->cfg)))
    return fail(ctx, MRR_EINVAL, "c_level_dev / b_level_dev is NULL or misaligned");
  if (c_level_dev == b_level_dev) return fail(ctx, MRR_EINVAL, "the blur cannot run in place");
  BlurParams bp = blur_params(ctx, g, lv);
  add_blur_slot(bp, lv, level, c_level_dev, b_level_dev);
  MRR_CUDA(ctx, launch_blur(bp, (cudaStream_t)stream));
  return MRR_OK;
}

uint64_t mrr_kernel_launches(void) { return mrr::launch_counter().load(); }

mrr_status mrr_batch_create(mrr_batch** out) {
  if (!out) return MRR_EINVAL;
  *out = nullptr;
  mrr_batch* b = new (std::nothrow) mrr_batch();
  if (!b) return MRR_ENOMEM;
  bool ok = cudaMalloc(&b->items_dev, MAX_BATCH * sizeof(BatchItem)) == cudaSuccess &&
            cudaMallocHost(&b->staging, MAX_BATCH * sizeof(BatchItem)) == cudaSuccess &&
            cudaMalloc(&b->queue_head, sizeof(uint32_t)) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->staging_done, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    mrr_batch_destroy(b);
    return MRR_ENOMEM;
  }
  *out = b;
  return MRR_OK;
}

void mrr_batch_destroy(mrr_batch* b) {
  if (!b) return;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  for (auto& t : b->topo)
    if (t.exec) cudaGraphExecDestroy(t.exec);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->staging_done) cudaEventDestroy(b->staging_done);
  cudaFree(b->items_dev);
  cudaFreeHost(b->staging);
  cudaFree(b->queue_head);
  delete b;
}

namespace {

mrr_status batch_fail(mrr_batch* b, mrr_status st, const char* msg) {
  b->err = msg;
  return st;
}

mrr_status check_batch(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, float* const* outs, int n) {
  if (!ctxs || !frames || n < 1 || n > MAX_BATCH) return batch_fail(b, MRR_EINVAL, "need 1..8 frames");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return batch_fail(b, MRR_EINVAL, "null context");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return batch_fail(b, MRR_EINVAL, "a context appears twice in the batch");
    mrr_status st = check_gbuffer(ctxs[k], &frames[k]);
    if (st != MRR_OK) return batch_fail(b, st, ctxs[k]->err.c_str());
    if (frames[k].width > ctxs[k]->pool_W || frames[k].height > ctxs[k]->pool_H)
      return batch_fail(b, MRR_EINVAL, "a frame exceeds its context's max size");
    if (ctxs[k]->cfg.pyramid_gathers)
      return batch_fail(b, MRR_EUNSUPPORTED, "pyramid gathers are not batched (single-frame calls only)");
    if (ctxs[k]->cfg.disjoint)
      return batch_fail(b, MRR_EUNSUPPORTED, "disjoint tiles are not batched (single-frame calls only)");
    if (outs && (!outs[k] || !aligned(outs[k], ctxs[k]->cfg.effect == MRR_SSGI ? 16 : 4)))
      return batch_fail(b, MRR_EINVAL, "output is NULL or misaligned");
  }
  return MRR_OK;
}

// The batch's launches: per-frame edges + masks, the item upload, one batched shading
// launch, per-frame merges.  outs == NULL stops after the shading launch (tuning).
mrr_status batch_launches(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, float* const* outs, int n,
                          int chunk, int grid, cudaStream_t s) {
  mrr_levels lv[MAX_BATCH];
  bool framed[MAX_BATCH];  // the frame path (at least two levels) or the staged one
  for (int k = 0; k < n; ++k) {
    mrr_ctx* ctx = ctxs[k];
    framed[k] = ctx->cfg.num_levels >= 2;
    mrr_status st;
    if (framed[k]) {
      if (!fits_pools(ctx, frames[k].width, frames[k].height))
        return batch_fail(b, MRR_EINVAL, "frame exceeds its context's max size");
      st = frame_masks(ctx, &frames[k], &lv[k], s, true);
    } else {
      st = edges_impl(ctx, &frames[k], ctx->edges, s);
      if (st != MRR_OK) return batch_fail(b, st, ctx->err.c_str());
      lv[k] = pool_levels(ctx, frames[k].width, frames[k].height);
      st = masks_impl(ctx, ctx->edges, &lv[k], s);
    }
    if (st != MRR_OK) return batch_fail(b, st, ctx->err.c_str());
  }
  for (int k = 0; k < n; ++k) {
    mrr_ctx* ctx = ctxs[k];
    BatchItem& it = b->staging[k];
    std::memset(&it, 0, sizeof it);
    it.p = make_shade_params(ctx, frames[k]);
    it.in = make_frame_in(frames[k]);
    it.precision = ctx->cfg.precision;
    for (int i = 0; i < ctx->cfg.num_levels; ++i) {
      if (!ctx->cfg.enabled[i] || (ctx->cfg.sample_levels && i > 0)) continue;
      const int q = it.lv.nlev++;
      it.lv.level[q] = i;
      it.lv.list[q] = ctx->worklist[i];
      it.lv.c[q] = ctx->cbuf[i];
      it.lv.Wi[q] = lv[k].width[i];
      it.lv.Hi[q] = lv[k].height[i];
      if (i == 0 && framed[k]) it.lv.compact |= 1 << q;
    }
    it.lv.counts = ctx->counts;
  }
  if (cudaMemcpyAsync(b->items_dev, b->staging, n * sizeof(BatchItem), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return batch_fail(b, MRR_ECUDA, "item upload");
  if (launch_shade_batch(b->items_dev, n, b->queue_head, chunk, grid, s) != cudaSuccess)
    return batch_fail(b, MRR_ECUDA, "batched shading launch");
  // sample-count levels above 0 are shaded per frame at full resolution
  for (int k = 0; k < n; ++k) {
    mrr_ctx* ctx = ctxs[k];
    if (!ctx->cfg.sample_levels) continue;
    for (int i = 1; i < ctx->cfg.num_levels; ++i) {
      if (!ctx->cfg.enabled[i]) continue;
      mrr_status st = shade_blocks_impl(ctx, frames[k], &lv[k], i, ctx->cbuf[i], s);
      if (st != MRR_OK) return batch_fail(b, st, ctx->err.c_str());
    }
  }
  if (outs) {
    for (int k = 0; k < n; ++k) {
      void* cm[MRR_MAX_LEVELS];
      mrr_status st = blur_pools(ctxs[k], &frames[k], &lv[k], cm, s);
      if (st == MRR_OK) st = merge_impl(ctxs[k], &lv[k], cm, outs[k], s, framed[k], frames[k].depth);
      if (st != MRR_OK) return batch_fail(b, st, ctxs[k]->err.c_str());
    }
  }
  return MRR_OK;
}

// Wait until the last item upload has read `staging` (never while capturing: a
// capturing thread may not wait on events).
mrr_status wait_staging(mrr_batch* b) {
  if (b->staging_pending) {
    if (cudaEventSynchronize(b->staging_done) != cudaSuccess) return batch_fail(b, MRR_ECUDA, "event sync");
    b->staging_pending = false;
  }
  return MRR_OK;
}

bool batch_key_matches(const mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, float* const* outs,
                       int n) {
  if (!b->graph_exec || b->key_n != n || b->key_chunk != b->chunk || b->key_grid != b->grid_mult) return false;
  for (int k = 0; k < n; ++k) {
    const mrr_gbuffer key = canonical_key(&frames[k]);
    if (b->key_ctx[k] != ctxs[k] || b->key_out[k] != outs[k] || std::memcmp(&key, &b->key_frame[k], sizeof key) != 0)
      return false;
  }
  return true;
}

}  // namespace

mrr_status mrr_render_batch(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, float* const* outs, int n,
                            void* stream) {
  if (!b) return MRR_EINVAL;
  if (!outs) return batch_fail(b, MRR_EINVAL, "outs is NULL");
  mrr_status st = check_batch(b, ctxs, frames, outs, n);
  if (st != MRR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = batch_grid_blocks() * b->grid_mult;
  if (!batch_key_matches(b, ctxs, frames, outs, n)) {
    if (b->graph_exec) {
      cudaGraphExecDestroy(b->graph_exec);
      b->graph_exec = nullptr;
    }
    st = wait_staging(b);
    if (st != MRR_OK) return st;
    if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return batch_fail(b, MRR_ECUDA, "begin capture");
    const uint64_t before = launch_counter().load();
    st = batch_launches(b, ctxs, frames, outs, n, b->chunk, grid, b->capture_stream);
    const uint64_t captured = launch_counter().load() - before;
    launch_counter().fetch_sub(captured);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
    if (st != MRR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return batch_fail(b, MRR_ECUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->graph_exec = nullptr;
      return batch_fail(b, MRR_ECUDA, "graph instantiate");
    }
    b->key_n = n;
    for (int k = 0; k < n; ++k) {
      b->key_ctx[k] = ctxs[k];
      b->key_out[k] = outs[k];
      b->key_frame[k] = canonical_key(&frames[k]);
    }
    b->key_chunk = b->chunk;
    b->key_grid = b->grid_mult;
    b->key_kernels = captured;
  }
  if (cudaGraphLaunch(b->graph_exec, s) != cudaSuccess) return batch_fail(b, MRR_ECUDA, "graph launch");
  count_launches((int)b->key_kernels);
  cudaEventRecord(b->staging_done, s);
  b->staging_pending = true;
  return MRR_OK;
}

const char* mrr_batch_last_error(mrr_batch* b) { return b ? b->err.c_str() : "no batch"; }

}  // extern "C"

// Serving: enqueue a batch with direct launches (no graph: every serving batch has new
// frames) on `stream`.  Not part of the C ABI.
mrr_status mrr_batch_enqueue_direct(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames,
                                    float* const* outs, int n, cudaStream_t stream) {
  mrr_status st = check_batch(b, ctxs, frames, outs, n);
  if (st != MRR_OK) return st;
  st = wait_staging(b);
  if (st != MRR_OK) return st;
  st = batch_launches(b, ctxs, frames, outs, n, b->chunk, batch_grid_blocks() * b->grid_mult, stream);
  if (st != MRR_OK) return st;
  cudaEventRecord(b->staging_done, stream);
  b->staging_pending = true;
  return MRR_OK;
}

// Serving: enqueue a batch as a CUDA graph keyed on its topology -- which contexts, in
// order, and the launch shape of the batched shading -- rather than on its pointers.
// Every request brings new frames and outputs, so the launches are captured afresh; when a
// graph of the same topology was instantiated before, the new capture is applied to it
// with cudaGraphExecUpdate (new kernel parameters and grid sizes for the same nodes), which
// costs far less than instantiating; a topology not seen before (or an update the driver
// refuses) is instantiated into the least recently used of TOPO_CACHE entries.
mrr_status mrr_batch_enqueue_graph(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames,
                                   float* const* outs, int n, cudaStream_t stream) {
  mrr_status st = check_batch(b, ctxs, frames, outs, n);
  if (st != MRR_OK) return st;
  st = wait_staging(b);
  if (st != MRR_OK) return st;
  mrr_batch::TopoGraph* hit = nullptr;
  for (auto& t : b->topo) {
    if (!t.exec || t.n != n || t.chunk != b->chunk || t.grid != b->grid_mult) continue;
    bool same = true;
    for (int k = 0; k < n && same; ++k) same = t.ctx[k] == ctxs[k];
    if (same) {
      hit = &t;
      break;
    }
  }
  if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return batch_fail(b, MRR_ECUDA, "begin capture");
  const uint64_t before = launch_counter().load();
  st = batch_launches(b, ctxs, frames, outs, n, b->chunk, batch_grid_blocks() * b->grid_mult, b->capture_stream);
  const uint64_t captured = launch_counter().load() - before;
  launch_counter().fetch_sub(captured);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
  if (st != MRR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return batch_fail(b, MRR_ECUDA, cudaGetErrorString(e));
  bool updated = false;
  if (hit) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(hit->exec, graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();  // an update the driver refuses leaves no sticky error
      cudaGraphExecDestroy(hit->exec);
      hit->exec = nullptr;
    }
  } else {
    hit = &b->topo[0];
    for (auto& t : b->topo)
      if (!t.exec || t.last_use < hit->last_use) hit = &t;
    if (hit->exec) cudaGraphExecDestroy(hit->exec);
    hit->exec = nullptr;
  }
  if (!updated) {
    e = cudaGraphInstantiate(&hit->exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      hit->exec = nullptr;
      return batch_fail(b, MRR_ECUDA, "graph instantiate");
    }
    ++b->graph_instantiations;
  } else {
    ++b->graph_updates;
  }
  cudaGraphDestroy(graph);
  hit->n = n;
  hit->chunk = b->chunk;
  hit->grid = b->grid_mult;
  for (int k = 0; k < n; ++k) hit->ctx[k] = ctxs[k];
  hit->kernels = captured;
  hit->last_use = ++b->topo_clock;
  if (cudaGraphLaunch(hit->exec, stream) != cudaSuccess) return batch_fail(b, MRR_ECUDA, "graph launch");
  count_launches((int)captured);
  cudaEventRecord(b->staging_done, stream);
  b->staging_pending = true;
  return MRR_OK;
}

void mrr_batch_graph_counts(const mrr_batch* b, uint64_t* instantiations, uint64_t* updates) {
  *instantiations = b ? b->graph_instantiations : 0;
  *updates = b ? b->graph_updates : 0;
}

extern "C" {

mrr_status mrr_batch_autotune(mrr_batch* b, mrr_ctx* const* ctxs, const mrr_gbuffer* frames, int n, void* stream,
                              mrr_batch_tuning* out) {
  if (!b) return MRR_EINVAL;
  mrr_status st = check_batch(b, ctxs, frames, nullptr, n);
  if (st != MRR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // masks and the item table once, then time the batched launch alone
  st = wait_staging(b);
  if (st != MRR_OK) return st;
  st = batch_launches(b, ctxs, frames, nullptr, n, b->chunk, batch_grid_blocks() * b->grid_mult, s);
  if (st != MRR_OK) return st;
  cudaEventRecord(b->staging_done, s);
  b->staging_pending = true;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return batch_fail(b, MRR_ECUDA, "event create");
  const int chunks[3] = {256, 1024, 4096};
  float best = 1e30f;
  int best_chunk = b->chunk, best_mult = b->grid_mult, cand = 0;
  for (int ci = 0; ci < 3; ++ci)
    for (int mult = 1; mult <= 2; ++mult) {
      float t[5];
      const int grid = batch_grid_blocks() * mult;
      for (int w = 0; w < 2; ++w) launch_shade_batch(b->items_dev, n, b->queue_head, chunks[ci], grid, s);
      for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, s);
        launch_shade_batch(b->items_dev, n, b->queue_head, chunks[ci], grid, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      std::sort(t, t + 5);
      ++cand;
      if (t[2] < best) {
        best = t[2];
        best_chunk = chunks[ci];
        best_mult = mult;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return batch_fail(b, MRR_ECUDA, "tuning launch");
  b->chunk = best_chunk;
  b->grid_mult = best_mult;
  if (out) {
    out->chunk = best_chunk;
    out->grid_multiplier = best_mult;
    out->shade_ms = best;
    out->candidates = cand;
  }
  return MRR_OK;
}

mrr_status mrr_autotune(mrr_ctx* ctx, const mrr_gbuffer* g, void* stream, mrr_tuning* out) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  if (g->width > ctx->pool_W || g->height > ctx->pool_H)
    return fail(ctx, MRR_EINVAL, "frame exceeds the context's max size");
  cudaStream_t s = (cudaStream_t)stream;
  const mrr_config& c = ctx->cfg;
  st = edges_impl(ctx, g, ctx->edges, s);
  if (st != MRR_OK) return st;
  mrr_levels lv = pool_levels(ctx, g->width, g->height);
  st = masks_impl(ctx, ctx->edges, &lv, s);
  if (st != MRR_OK) return st;
  ShadeParams p = make_shade_params(ctx, *g);
  ShadeLevels sl;
  std::memset(&sl, 0, sizeof sl);
  for (int i = 0; i < c.num_levels; ++i) {
    if (!c.enabled[i]) continue;
    const int k = sl.nlev++;
    sl.level[k] = i;
    sl.list[k] = ctx->worklist[i];
    sl.c[k] = ctx->cbuf[i];
    sl.Wi[k] = lv.width[i];
    sl.Hi[k] = lv.height[i];
  }
  sl.counts = ctx->counts;
  cudaEvent_t e0, e1;
  MRR_CUDA(ctx, cudaEventCreate(&e0));
  MRR_CUDA(ctx, cudaEventCreate(&e1));
  // a buffer larger than L2, rewritten before every timed launch so each one starts cold
  const size_t flush_bytes = (size_t)256 << 20;
  void* flush = nullptr;
  if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) flush = nullptr;
  auto median_ms = [&](auto&& launch) -> float {
    float t[5];
    for (int w = 0; w < 2; ++w) launch();
    for (int r = 0; r < 5; ++r) {
      if (flush) cudaMemsetAsync(flush, r, flush_bytes, s);
      cudaEventRecord(e0, s);
      launch();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[r], e0, e1);
    }
    std::sort(t, t + 5);
    return t[2];
  };
  const FrameIn in = make_frame_in(*g);
  const bool ssao = c.effect == MRR_SSAO;
  const int lanes_opts[3] = {1, 2, 4};
  int best_lanes = ctx->split_texel, best_mult = 1, cand = 0;
  float best = 1e30f;
  for (int li = 0; li < 3; ++li) {
    const int lanes = lanes_opts[li];
    if (!ssao && lanes != 1) continue;
    if (c.lanes_per_texel && lanes != c.lanes_per_texel) continue;
    for (int mult = 1; mult <= 4; mult *= 2) {
      const float ms = median_ms([&] {
        launch_shade_levels(p, in, c.precision, sl, shade_grid_blocks() * mult, lanes, s);
      });
      ++cand;
      if (ms < best) {
        best = ms;
        best_lanes = lanes;
        best_mult = mult;
      }
    }
  }
  int best_pix = ctx->split_pixel;
  float best_full = 1e30f;
  float* tmp = nullptr;  // the full-resolution kernel's output while it is timed
  MRR_CUDA(ctx, cudaMalloc(&tmp, (size_t)g->width * g->height * sizeof(float) * channels(c)));
  for (int li = 0; li < 3; ++li) {
    const int lanes = lanes_opts[li];
    if (!ssao && lanes != 1) continue;
    if (c.lanes_per_pixel && lanes != c.lanes_per_pixel) continue;
    const float ms = median_ms([&] { launch_shade_full(p, in, c.precision, tmp, lanes, s); });
    ++cand;
    if (ms < best_full) {
      best_full = ms;
      best_pix = lanes;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  cudaFree(flush);
  MRR_CUDA(ctx, cudaGetLastError());
  ctx->split_texel = best_lanes;
  ctx->split_pixel = best_pix;
  ctx->shade_grid = shade_grid_blocks() * best_mult;
  for (int e = 0; e < 2; ++e)  // the captured launches used the old settings
    if (ctx->graph_exec[e]) {
      cudaGraphExecDestroy(ctx->graph_exec[e]);
      ctx->graph_exec[e] = nullptr;
    }
  if (out) {
    out->lanes_per_texel = best_lanes;
    out->grid_multiplier = best_mult;
    out->lanes_per_pixel = best_pix;
    out->shade_levels_ms = best;
    out->shade_full_ms = best_full;
    out->candidates = cand;
  }
  return MRR_OK;
}

mrr_status mrr_upsample_merge(mrr_ctx* ctx, const mrr_levels* lv, void* const* c_levels_dev, float* out_dev,
                              void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_levels(ctx, lv, false);
  if (st != MRR_OK) return st;
  if (!c_levels_dev || !out_dev) return fail(ctx, MRR_EINVAL, "c_levels_dev / out_dev is NULL");
  for (int i = 0; i < ctx->cfg.num_levels; ++i)
    if (ctx->cfg.enabled[i] && (!c_levels_dev[i] || !aligned(c_levels_dev[i], cbytes(ctx->cfg))))
      return fail(ctx, MRR_EINVAL, "sub-image %d is NULL or misaligned", i);
  if (!aligned(out_dev, ctx->cfg.effect == MRR_SSGI ? 16 : 4)) return fail(ctx, MRR_EINVAL, "out_dev misaligned");
  if (ctx->cfg.merge_mode == 1 && !fits_pools(ctx, lv->width[0], lv->height[0]))
    return fail(ctx, MRR_EINVAL, "step-wise blending: frame %dx%d exceeds the context's max size", lv->width[0],
                lv->height[0]);
  if (ctx->cfg.merge_mode == 2 && !ctx->cfg.sample_levels)
    return fail(ctx, MRR_EINVAL, "the bilateral merge needs the frame's depth: mrr_upsample_merge_bilateral");
  return merge_impl(ctx, lv, c_levels_dev, out_dev, (cudaStream_t)stream);
}

mrr_status mrr_upsample_merge_bilateral(mrr_ctx* ctx, const mrr_gbuffer* g, const mrr_levels* lv,
                                        void* const* c_levels_dev, float* out_dev, void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  st = check_levels(ctx, lv, false);
  if (st != MRR_OK) return st;
  if (ctx->cfg.merge_mode != 2 || ctx->cfg.sample_levels)
    return fail(ctx, MRR_EINVAL, "mrr_upsample_merge_bilateral needs merge_mode 2");
  if (lv->width[0] != g->width || lv->height[0] != g->height)
    return fail(ctx, MRR_EINVAL, "levels are for %dx%d, frame is %dx%d", lv->width[0], lv->height[0], g->width,
                g->height);
  if (!c_levels_dev || !out_dev) return fail(ctx, MRR_EINVAL, "c_levels_dev / out_dev is NULL");
  for (int i = 0; i < ctx->cfg.num_levels; ++i)
    if (ctx->cfg.enabled[i] && (!c_levels_dev[i] || !aligned(c_levels_dev[i], cbytes(ctx->cfg))))
      return fail(ctx, MRR_EINVAL, "sub-image %d is NULL or misaligned", i);
  if (!aligned(out_dev, ctx->cfg.effect == MRR_SSGI ? 16 : 4)) return fail(ctx, MRR_EINVAL, "out_dev misaligned");
  return merge_impl(ctx, lv, c_levels_dev, out_dev, (cudaStream_t)stream, false, g->depth);
}

mrr_status mrr_render(mrr_ctx* ctx, const mrr_gbuffer* g, float* out_dev, void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  if (g->width > ctx->pool_W || g->height > ctx->pool_H)
    return fail(ctx, MRR_EINVAL, "frame %dx%d exceeds the context's max size %dx%d", g->width, g->height,
                ctx->pool_W, ctx->pool_H);
  if (!out_dev || !aligned(out_dev, ctx->cfg.effect == MRR_SSGI ? 16 : 4))
    return fail(ctx, MRR_EINVAL, "out_dev is NULL or misaligned");
  return render_impl(ctx, g, out_dev, (cudaStream_t)stream);
}

mrr_status mrr_trace_shading(mrr_ctx* ctx, void* event_begin, void* event_end) {
  if (!ctx) return MRR_EINVAL;
  if ((event_begin == nullptr) != (event_end == nullptr))
    return fail(ctx, MRR_EINVAL, "trace events: both or neither");
  ctx->trace_begin = (cudaEvent_t)event_begin;
  ctx->trace_end = (cudaEvent_t)event_end;
  return MRR_OK;
}

mrr_status mrr_render_full(mrr_ctx* ctx, const mrr_gbuffer* g, float* out_dev, void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, g);
  if (st != MRR_OK) return st;
  if (!out_dev || !aligned(out_dev, ctx->cfg.effect == MRR_SSGI ? 16 : 4))
    return fail(ctx, MRR_EINVAL, "out_dev is NULL or misaligned");
  ShadeParams p = make_shade_params(ctx, *g);
  MRR_CUDA(ctx, launch_shade_full(p, make_frame_in(*g), ctx->cfg.precision, out_dev, ctx->split_pixel,
                                  (cudaStream_t)stream));
  return MRR_OK;
}

mrr_status mrr_render_host_async(mrr_ctx* ctx, const mrr_gbuffer* gh, float* out_host) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, gh, false);
  if (st != MRR_OK) return st;
  if (!out_host) return fail(ctx, MRR_EINVAL, "out_host is NULL");
  const mrr_config& c = ctx->cfg;
  const int W = gh->width, H = gh->height;
  if (W > ctx->pool_W || H > ctx->pool_H) return fail(ctx, MRR_EINVAL, "frame exceeds the context's max size");
  const size_t npx_max = (size_t)ctx->pool_W * ctx->pool_H, npx = (size_t)W * H;
  const size_t nbytes = c.precision == MRR_FP16 ? 8 : 16;
  const size_t sm_bytes = c.effect == MRR_SSM
                              ? (size_t)gh->shadow_size * gh->shadow_size * sizeof(float)
                              : 0;
  for (cudaStream_t* sp : {&ctx->s_in, &ctx->s_comp, &ctx->s_out})
    if (!*sp) MRR_CUDA(ctx, cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking));
  mrr_ctx::HostSet& hs = ctx->hset[ctx->hset_next];
  if (!hs.depth) {
    MRR_CUDA(ctx, cudaMalloc(&hs.depth, npx_max * sizeof(float)));
    MRR_CUDA(ctx, cudaMalloc(&hs.normal, npx_max * nbytes));
    MRR_CUDA(ctx, cudaMalloc(&hs.out, npx_max * sizeof(float) * channels(c)));
    if (c.effect == MRR_SSGI) MRR_CUDA(ctx, cudaMalloc(&hs.color, npx_max * 8));
    for (cudaEvent_t* ev : {&hs.loaded, &hs.rendered, &hs.done})
      MRR_CUDA(ctx, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  }
  if (sm_bytes > hs.smap_bytes) {
    // the set's previous frame may still read its shadow map
    if (hs.used) MRR_CUDA(ctx, cudaEventSynchronize(hs.rendered));
    cudaFree(hs.smap);
    hs.smap = nullptr;
    hs.smap_bytes = 0;
    MRR_CUDA(ctx, cudaMalloc(&hs.smap, sm_bytes));
    hs.smap_bytes = sm_bytes;
  }
  // uploads into the set wait until its previous frame was rendered (inputs read)
  if (hs.used) MRR_CUDA(ctx, cudaStreamWaitEvent(ctx->s_in, hs.rendered, 0));
  mrr_gbuffer g = *gh;
  MRR_CUDA(ctx, cudaMemcpyAsync(hs.depth, gh->depth, npx * sizeof(float), cudaMemcpyHostToDevice, ctx->s_in));
  MRR_CUDA(ctx, cudaMemcpyAsync(hs.normal, gh->normal, npx * nbytes, cudaMemcpyHostToDevice, ctx->s_in));
  g.depth = hs.depth;
  g.normal = hs.normal;
  if (c.effect == MRR_SSGI) {
    MRR_CUDA(ctx, cudaMemcpyAsync(hs.color, gh->color, npx * 8, cudaMemcpyHostToDevice, ctx->s_in));
    g.color = hs.color;
  }
  if (c.effect == MRR_SSM) {
    MRR_CUDA(ctx, cudaMemcpyAsync(hs.smap, gh->shadow_map, sm_bytes, cudaMemcpyHostToDevice, ctx->s_in));
    g.shadow_map = hs.smap;
  }
  MRR_CUDA(ctx, cudaEventRecord(hs.loaded, ctx->s_in));
  // rendering waits for the inputs and for the set's previous image to be downloaded
  MRR_CUDA(ctx, cudaStreamWaitEvent(ctx->s_comp, hs.loaded, 0));
  if (hs.used) MRR_CUDA(ctx, cudaStreamWaitEvent(ctx->s_comp, hs.done, 0));
  st = render_impl(ctx, &g, hs.out, ctx->s_comp);
  if (st != MRR_OK) return st;
  MRR_CUDA(ctx, cudaEventRecord(hs.rendered, ctx->s_comp));
  MRR_CUDA(ctx, cudaStreamWaitEvent(ctx->s_out, hs.rendered, 0));
  MRR_CUDA(ctx, cudaMemcpyAsync(out_host, hs.out, npx * sizeof(float) * channels(c), cudaMemcpyDeviceToHost,
                                ctx->s_out));
  MRR_CUDA(ctx, cudaEventRecord(hs.done, ctx->s_out));
  hs.used = true;
  ctx->hset_next ^= 1;
  return MRR_OK;
}

mrr_status mrr_render_host_wait(mrr_ctx* ctx) {
  if (!ctx) return MRR_EINVAL;
  for (cudaStream_t st : {ctx->s_in, ctx->s_comp, ctx->s_out})
    if (st) MRR_CUDA(ctx, cudaStreamSynchronize(st));
  return MRR_OK;
}

mrr_status mrr_render_host(mrr_ctx* ctx, const mrr_gbuffer* gh, float* out_host, void* stream) {
  if (!ctx) return MRR_EINVAL;
  mrr_status st = check_gbuffer(ctx, gh, false);
  if (st != MRR_OK) return st;
  if (!out_host) return fail(ctx, MRR_EINVAL, "out_host is NULL");
  const mrr_config& c = ctx->cfg;
  const int W = gh->width, H = gh->height;
  if (W > ctx->pool_W || H > ctx->pool_H) return fail(ctx, MRR_EINVAL, "frame exceeds the context's max size");
  const size_t npx_max = (size_t)ctx->pool_W * ctx->pool_H, npx = (size_t)W * H;
  const size_t nbytes = c.precision == MRR_FP16 ? 8 : 16;
  if (!ctx->h_depth) {
    MRR_CUDA(ctx, cudaMalloc(&ctx->h_depth, npx_max * sizeof(float)));
    MRR_CUDA(ctx, cudaMalloc(&ctx->h_normal, npx_max * nbytes));
    MRR_CUDA(ctx, cudaMalloc(&ctx->h_out, npx_max * sizeof(float) * channels(c)));
    if (c.effect == MRR_SSGI) MRR_CUDA(ctx, cudaMalloc(&ctx->h_color, npx_max * 8));
  }
  const size_t sm_bytes = c.effect == MRR_SSM
                              ? (size_t)gh->shadow_size * gh->shadow_size * sizeof(float)
                              : 0;
  if (sm_bytes > ctx->h_smap_bytes) {
    cudaFree(ctx->h_smap);
    ctx->h_smap = nullptr;
    ctx->h_smap_bytes = 0;
    MRR_CUDA(ctx, cudaMalloc(&ctx->h_smap, sm_bytes));
    ctx->h_smap_bytes = sm_bytes;
  }
  cudaStream_t s = (cudaStream_t)stream;
  mrr_gbuffer g = *gh;
  MRR_CUDA(ctx, cudaMemcpyAsync(ctx->h_depth, gh->depth, npx * sizeof(float), cudaMemcpyHostToDevice, s));
  MRR_CUDA(ctx, cudaMemcpyAsync(ctx->h_normal, gh->normal, npx * nbytes, cudaMemcpyHostToDevice, s));
  g.depth = ctx->h_depth;
  g.normal = ctx->h_normal;
  if (c.effect == MRR_SSGI) {
    MRR_CUDA(ctx, cudaMemcpyAsync(ctx->h_color, gh->color, npx * 8, cudaMemcpyHostToDevice, s));
    g.color = ctx->h_color;
  }
  if (c.effect == MRR_SSM) {
    MRR_CUDA(ctx, cudaMemcpyAsync(ctx->h_smap, gh->shadow_map, sm_bytes, cudaMemcpyHostToDevice, s));
    g.shadow_map = ctx->h_smap;
  }
  st = render_impl(ctx, &g, ctx->h_out, s);
  if (st != MRR_OK) return st;
  MRR_CUDA(ctx, cudaMemcpyAsync(out_host, ctx->h_out, npx * sizeof(float) * channels(c), cudaMemcpyDeviceToHost, s));
  MRR_CUDA(ctx, cudaStreamSynchronize(s));
  return MRR_OK;
}

}  // extern "C"
