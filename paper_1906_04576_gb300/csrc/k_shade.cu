// k_shade.cu -- rendering the sub-images (Sec. 3.2 / Sec. 4.1) and the naive
// full-resolution rendering the paper compares against (Sec. 5).
//
// shade_levels_kernel: a persistent grid strides over the concatenation of the work
//   lists of one or more levels (their lengths are read on the device, so the launch
//   needs no host synchronisation).  Consecutive lane groups take consecutive list
//   entries, i.e. neighbouring texels of one row, so the gathers of one sample index land
//   close together and every lane has real work -- the GPU counterpart of the stencil
//   test.  For SSAO, SPLIT lanes share a texel and split its samples (the occlusion count
//   is an integer, so the split is exact); SSM and SSGI accumulate floats in sample order
//   and use one lane per texel.
// shade_full_kernel: one lane group per pixel over 2-D tiles of 8 rows.
// shade_blocks_kernel: sample-count levels -- every pixel of a listed texel's block at
//   full resolution, with the level's thinned sample tables.
// pyramid_kernel: the point-sampled depth of the levels above 0 that SSAO's gathers read
//   with pyramid gathers (a separate instantiation of shade_levels_kernel).
// Both evaluate the same effect function at the same full-resolution pixel, so a level
// texel's value equals full-resolution shading at its sample pixel bit for bit.
#include "mrr_internal.cuh"
#include "shade_common.cuh"

namespace mrr {

namespace {

constexpr int SHADE_THREADS = 256;

// FIX: the SSAO variant compiled for 64 samples.  Its sample loop unrolls completely and
// every table entry becomes a constant operand instead of an indexed load.  Resident
// CTAs per SM the register allocation must allow: left at 2 CTAs (128 registers) the
// compiler hoists the loads of many samples at once and the kernel loses occupancy,
// while 6 CTAs (42 registers) keep 48 warps per SM in flight -- the fastest of 3 to 7 at
// 1920x1080 and 3840x2160.
constexpr int FIX_SSAO = 64;
constexpr int shade_min_blocks(bool FIX) { return FIX ? 6 : 2; }

inline bool fixed_counts(const ShadeParams& p) { return p.effect == MRR_SSAO && p.samples == FIX_SSAO; }

template <int EFFECT, typename NT, typename SMT, int SPLIT, bool PYR = false, bool FIX = false>
__device__ __forceinline__ float3 effect_at(const ShadeParams& p, const FrameIn& in, int x, int y, bool valid,
                                            const GatherDepth gd = GatherDepth{}) {
  if (EFFECT == MRR_SSAO) {
    return make_float3(ssao_at<NT, SPLIT, PYR, FIX ? FIX_SSAO : 0>(p, in.depth, (const NT*)in.normal, x, y, valid, gd), 0.f, 0.f);
  } else if (EFFECT == MRR_SSM) {
    return valid ? make_float3(ssm_at<SMT>(p, in.depth, (const SMT*)in.smap, x, y), 0.f, 0.f)
                 : make_float3(0.f, 0.f, 0.f);
  } else {
    return valid ? ssgi_at<NT>(p, in.depth, (const NT*)in.normal, in.color, x, y) : make_float3(0.f, 0.f, 0.f);
  }
}

// Store an effect value into a sub-image texel / output pixel.
template <int EFFECT>
__device__ __forceinline__ void store_value(void* c, size_t i, float3 v, bool half_store) {
  if (EFFECT == MRR_SSGI) {
    if (half_store) {
      half4 h;
      h.x = __float2half_rn(v.x);
      h.y = __float2half_rn(v.y);
      h.z = __float2half_rn(v.z);
      h.w = __float2half_rn(0.0f);
      reinterpret_cast<half4*>(c)[i] = h;
    } else {
      reinterpret_cast<float4*>(c)[i] = make_float4(v.x, v.y, v.z, 0.0f);
    }
  } else {
    if (half_store)
      reinterpret_cast<__half*>(c)[i] = __float2half_rn(v.x);
    else
      reinterpret_cast<float*>(c)[i] = v.x;
  }
}

template <int EFFECT, typename NT, typename SMT, int SPLIT, bool PYR = false, bool FIX = false>
__global__ void __launch_bounds__(SHADE_THREADS, shade_min_blocks(FIX))
    shade_levels_kernel(ShadeParams p, FrameIn in, ShadeLevels lv, int half_store) {
  // per-level descriptors in shared memory (indexed by a runtime level slot)
  __shared__ uint32_t s_pre[MRR_MAX_LEVELS + 1];
  __shared__ const uint32_t* s_list[MRR_MAX_LEVELS];
  __shared__ void* s_c[MRR_MAX_LEVELS];
  __shared__ int s_lvl[MRR_MAX_LEVELS], s_W[MRR_MAX_LEVELS], s_H[MRR_MAX_LEVELS];
  __shared__ const float* s_pyr[MRR_MAX_LEVELS];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    s_pre[0] = 0;
#pragma unroll
    for (int k = 0; k < MRR_MAX_LEVELS; ++k) {
      if (k >= lv.nlev) break;
      acc += min(__ldg(lv.counts + lv.level[k]), (uint32_t)lv.Wi[k] * (uint32_t)lv.Hi[k]);
      s_pre[k + 1] = acc;
      s_list[k] = lv.list[k];
      s_c[k] = lv.c[k];
      s_lvl[k] = lv.level[k];
      s_W[k] = lv.Wi[k];
      s_H[k] = lv.Hi[k];
      if (PYR) s_pyr[k] = lv.level[k] > 0 ? lv.pyr[k] : in.depth;
    }
  }
  __syncthreads();
  const int nlev = lv.nlev;
  const uint32_t total = s_pre[nlev];
  const uint32_t lanes = total * SPLIT;
  const int W = p.v.W, H = p.v.H;
  const int sub = threadIdx.x & (SPLIT - 1);
  for (uint32_t base = blockIdx.x * SHADE_THREADS; base < lanes; base += gridDim.x * SHADE_THREADS) {
    const uint32_t g = (base + threadIdx.x) / SPLIT;
    bool valid = g < total;
    int k = 0, x = 0, y = 0, qx = 0, qy = 0;
    if (valid) {
      while (k + 1 < nlev && g >= s_pre[k + 1]) ++k;
      const int i = s_lvl[k];
      const uint32_t e = __ldg(s_list[k] + (g - s_pre[k]));
      qx = (int)(e & 0xFFFFu);
      qy = (int)(e >> 16);
      valid = qx < s_W[k] && qy < s_H[k];  // skip anything that is not a texel of the level
      const int o = i == 0 ? 0 : (1 << (i - 1));
      x = min((qx << i) + o, W - 1);
      y = min((qy << i) + o, H - 1);
    }
    GatherDepth gd{};
    if (PYR) {  // the slot's level (0: full resolution), for every lane of the warp
      const int lvl = valid ? s_lvl[k] : 0;
      gd.base = valid ? s_pyr[k] : in.depth;
      gd.shift = lvl;
      gd.width = lvl > 0 ? s_W[k] : W;
    }
    const float3 v = effect_at<EFFECT, NT, SMT, SPLIT, PYR, FIX>(p, in, x, y, valid, gd);
    if (valid && sub == 0)
      store_value<EFFECT>(s_c[k], ((lv.compact >> k) & 1) ? (size_t)(g - s_pre[k]) : (size_t)qy * s_W[k] + qx, v,
                          half_store != 0);
  }
}

template <int EFFECT, typename NT, typename SMT, int SPLIT, bool FIX = false>
__global__ void __launch_bounds__(256, shade_min_blocks(FIX))
    shade_full_kernel(ShadeParams p, FrameIn in, float* __restrict__ out) {
  // block = 32 x 8 lanes; a warp row covers 32 / SPLIT consecutive pixels
  const int x = blockIdx.x * (32 / SPLIT) + (int)threadIdx.x / SPLIT;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const bool valid = x < p.v.W && y < p.v.H;
  const float3 v = effect_at<EFFECT, NT, SMT, SPLIT, false, FIX>(p, in, valid ? x : 0, valid ? y : 0, valid);
  if (valid && (threadIdx.x & (SPLIT - 1)) == 0) store_value<EFFECT>(out, (size_t)y * p.v.W + x, v, false);
}

// Sample-count levels (Sec. 6): one lane per full-resolution pixel of each listed texel's
// block, with the level's thinned sample tables in p; lanes past the end (or on an entry
// that is not a texel of the level, or a pixel past the image) shade nothing.
template <int EFFECT, typename NT, typename SMT>
__global__ void __launch_bounds__(SHADE_THREADS, 2) shade_blocks_kernel(ShadeParams p, FrameIn in, BlockLevel b,
                                                                     int half_store) {
  const int W = p.v.W, H = p.v.H, i = b.level, B = 1 << b.level;
  const uint32_t n = min(__ldg(b.count), (uint32_t)b.Wi * (uint32_t)b.Hi);
  const uint32_t total = n << (2 * i);
  for (uint32_t base = blockIdx.x * SHADE_THREADS; base < total; base += gridDim.x * SHADE_THREADS) {
    const uint32_t g = base + threadIdx.x;
    bool valid = g < total;
    int x = 0, y = 0;
    if (valid) {
      const uint32_t e = __ldg(b.list + (g >> (2 * i)));
      const int qx = (int)(e & 0xFFFFu), qy = (int)(e >> 16);
      const uint32_t sub = g & ((1u << (2 * i)) - 1u);
      const int px = qx * B + (int)(sub & (uint32_t)(B - 1)), py = qy * B + (int)(sub >> i);
      valid = qx < b.Wi && qy < b.Hi && px < W && py < H;
      if (valid) {
        x = px;
        y = py;
      }
    }
    const float3 v = effect_at<EFFECT, NT, SMT, 1>(p, in, x, y, valid);
    if (valid) store_value<EFFECT>(b.c, (size_t)y * W + x, v, half_store != 0);
  }
}

// Point-sampled depth of the levels above 0 for pyramid gathers: out[k][Q] = depth[s_i(Q)].
__global__ void __launch_bounds__(256) pyramid_kernel(PyramidParams p) {
  uint32_t n[MRR_MAX_LEVELS], total = 0;
#pragma unroll
  for (int k = 0; k < MRR_MAX_LEVELS; ++k) {
    n[k] = k < p.nlev ? (uint32_t)p.Wi[k] * (uint32_t)p.Hi[k] : 0u;
    total += n[k];
  }
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int k = 0;
    uint32_t e = g;
#pragma unroll
    for (int j = 0; j < MRR_MAX_LEVELS - 1; ++j)
      if (k == j && e >= n[j]) {
        e -= n[j];
        k = j + 1;
      }
    const int i = p.level[k], Wi = p.Wi[k];
    const int qy = (int)(e / (uint32_t)Wi), qx = (int)(e - (uint32_t)qy * Wi);
    const int o = i == 0 ? 0 : 1 << (i - 1);
    const int sx = min(qx * (1 << i) + o, p.W - 1), sy = min(qy * (1 << i) + o, p.H - 1);
    p.out[k][e] = __ldg(p.depth + (size_t)sy * p.W + sx);
  }
}

// Resident CTAs of one instantiation (SMs x CTAs per SM), computed once per instantiation.
template <typename K> int resident_blocks(K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, SHADE_THREADS, 0);
  return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

// `grid_mult` x the resident CTAs of this very instantiation: a persistent grid that is
// one full wave (or a whole number of waves), never 1.2.
template <int EFFECT, typename NT, typename SMT, int SPLIT>
void launch_levels_t(const ShadeParams& p, const FrameIn& in, const ShadeLevels& lv, int half_store, int grid_mult,
                     cudaStream_t s) {
  if (EFFECT == MRR_SSAO && lv.pyramid) {
    static const int resident_p = resident_blocks(shade_levels_kernel<EFFECT, NT, SMT, SPLIT, true>);
    shade_levels_kernel<EFFECT, NT, SMT, SPLIT, true><<<resident_p * grid_mult, SHADE_THREADS, 0, s>>>(p, in, lv,
                                                                                                     half_store);
    return;
  }
  if constexpr (EFFECT == MRR_SSAO && SPLIT == 1) {
    if (fixed_counts(p)) {
      static const int resident_f = resident_blocks(shade_levels_kernel<EFFECT, NT, SMT, SPLIT, false, true>);
      shade_levels_kernel<EFFECT, NT, SMT, SPLIT, false, true><<<resident_f * grid_mult, SHADE_THREADS, 0, s>>>(
          p, in, lv, half_store);
      return;
    }
  }
  static const int resident = resident_blocks(shade_levels_kernel<EFFECT, NT, SMT, SPLIT>);
  shade_levels_kernel<EFFECT, NT, SMT, SPLIT><<<resident * grid_mult, SHADE_THREADS, 0, s>>>(p, in, lv, half_store);
}

template <int EFFECT, typename NT, typename SMT, int SPLIT>
void launch_full_t(const ShadeParams& p, const FrameIn& in, float* out, cudaStream_t s) {
  dim3 block(32, 8), grid((p.v.W + 32 / SPLIT - 1) / (32 / SPLIT), (p.v.H + 7) / 8);
  if constexpr (EFFECT == MRR_SSAO && SPLIT == 1) {
    if (fixed_counts(p)) {
      shade_full_kernel<EFFECT, NT, SMT, SPLIT, true><<<grid, block, 0, s>>>(p, in, out);
      return;
    }
  }
  shade_full_kernel<EFFECT, NT, SMT, SPLIT><<<grid, block, 0, s>>>(p, in, out);
}

template <int EFFECT, typename NT, typename SMT>
void launch_blocks_t(const ShadeParams& p, const FrameIn& in, const BlockLevel& b, int half_store, int grid_mult,
                     cudaStream_t s) {
  static const int resident = resident_blocks(shade_blocks_kernel<EFFECT, NT, SMT>);
  shade_blocks_kernel<EFFECT, NT, SMT><<<resident * grid_mult, SHADE_THREADS, 0, s>>>(p, in, b, half_store);
}

template <typename NT, typename SMT>
void blocks_dispatch(const ShadeParams& p, const FrameIn& in, const BlockLevel& b, int half_store, int grid,
                     cudaStream_t s) {
  switch (p.effect) {
    case MRR_SSAO: launch_blocks_t<MRR_SSAO, NT, SMT>(p, in, b, half_store, grid, s); break;
    case MRR_SSM: launch_blocks_t<MRR_SSM, NT, SMT>(p, in, b, half_store, grid, s); break;
    default: launch_blocks_t<MRR_SSGI, NT, SMT>(p, in, b, half_store, grid, s); break;
  }
}

template <typename NT, typename SMT>
void levels_dispatch(const ShadeParams& p, const FrameIn& in, const ShadeLevels& lv, int half_store, int grid,
                     int split, cudaStream_t s) {  // grid: multiple of the resident CTAs
  switch (p.effect) {
    case MRR_SSAO:
      if (split >= 4) launch_levels_t<MRR_SSAO, NT, SMT, 4>(p, in, lv, half_store, grid, s);
      else if (split == 2) launch_levels_t<MRR_SSAO, NT, SMT, 2>(p, in, lv, half_store, grid, s);
      else launch_levels_t<MRR_SSAO, NT, SMT, 1>(p, in, lv, half_store, grid, s);
      break;
    case MRR_SSM:
      launch_levels_t<MRR_SSM, NT, SMT, 1>(p, in, lv, half_store, grid, s);
      break;
    default:
      launch_levels_t<MRR_SSGI, NT, SMT, 1>(p, in, lv, half_store, grid, s);
      break;
  }
}

template <typename NT, typename SMT>
void full_dispatch(const ShadeParams& p, const FrameIn& in, float* out, int split, cudaStream_t s) {
  switch (p.effect) {
    case MRR_SSAO:
      if (split >= 4) launch_full_t<MRR_SSAO, NT, SMT, 4>(p, in, out, s);
      else if (split == 2) launch_full_t<MRR_SSAO, NT, SMT, 2>(p, in, out, s);
      else launch_full_t<MRR_SSAO, NT, SMT, 1>(p, in, out, s);
      break;
    case MRR_SSM:
      launch_full_t<MRR_SSM, NT, SMT, 1>(p, in, out, s);
      break;
    default:
      launch_full_t<MRR_SSGI, NT, SMT, 1>(p, in, out, s);
      break;
  }
}

}  // namespace

__global__ void check_reciprocal_kernel(uint32_t first, uint32_t last, unsigned long long* bad) {
  unsigned long long n = 0;
  for (uint64_t b = (uint64_t)first + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b <= last;
       b += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((uint32_t)b);
    const float2 two = rcp_rn2(make_float2(x, -x));
    const uint32_t want = __float_as_uint(__frcp_rn(x));
    n += (__float_as_uint(rcp_rn(x)) != want) + (__float_as_uint(two.x) != want) +
         (__float_as_uint(two.y) != (want ^ 0x80000000u));
  }
  if (n) atomicAdd(bad, n);
}

cudaError_t launch_check_reciprocal(uint32_t first, uint32_t last, unsigned long long* bad, cudaStream_t s) {
  check_reciprocal_kernel<<<152 * 16, 256, 0, s>>>(first, last, bad);
  count_launches(1);
  return cudaGetLastError();
}

std::atomic<uint64_t>& launch_counter() {
  static std::atomic<uint64_t> n{0};
  return n;
}

int shade_grid_blocks() { return 1; }  // the launch scales the resident CTAs of its own variant

cudaError_t launch_shade_levels(const ShadeParams& p, const FrameIn& in, int precision, const ShadeLevels& lv,
                                int grid, int split, cudaStream_t s) {
  if (precision == MRR_FP16) levels_dispatch<half4, float>(p, in, lv, 1, grid, split, s);
  else levels_dispatch<float4, float>(p, in, lv, 0, grid, split, s);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pyramid(const PyramidParams& p, cudaStream_t s) {
  if (p.nlev == 0) return cudaSuccess;
  pyramid_kernel<<<152 * 8, 256, 0, s>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_shade_blocks(const ShadeParams& p, const FrameIn& in, int precision, const BlockLevel& b,
                                int grid_mult, cudaStream_t s) {
  if (precision == MRR_FP16) blocks_dispatch<half4, float>(p, in, b, 1, grid_mult, s);
  else blocks_dispatch<float4, float>(p, in, b, 0, grid_mult, s);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_shade_full(const ShadeParams& p, const FrameIn& in, int precision, float* out, int split,
                              cudaStream_t s) {
  if (precision == MRR_FP16) full_dispatch<half4, float>(p, in, out, split, s);
  else full_dispatch<float4, float>(p, in, out, split, s);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
