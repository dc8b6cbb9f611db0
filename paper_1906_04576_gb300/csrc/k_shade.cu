// k_shade.cu -- rendering the sub-images (Sec. 3.2 / Sec. 4.1) and the naive
// full-resolution rendering the paper compares against (Sec. 5).
//
// shade_levels_kernel: a persistent grid strides over the concatenation of the work
//   lists of one or more levels (their lengths are read on the device, so the launch
//   needs no host synchronisation).  Consecutive lanes take consecutive list entries,
//   i.e. neighbouring texels of one row, so the gathers of one sample index land close
//   together and every lane has real work -- the GPU counterpart of the stencil test.
// shade_full_kernel: one thread per pixel over 32x8 tiles.
// Both evaluate the same effect function at the same full-resolution pixel, so a
// level texel's value equals full-resolution shading at its sample pixel bit for bit.
#include "mrr_internal.cuh"
#include "shade_common.cuh"

namespace mrr {

namespace {

constexpr int SHADE_THREADS = 256;

template <int EFFECT, typename NT, typename SMT>
__device__ __forceinline__ float3 effect_at(const ShadeParams& p, const FrameIn& in, int x, int y) {
  if (EFFECT == MRR_SSAO) {
    return make_float3(ssao_at<NT>(p, in.depth, (const NT*)in.normal, x, y), 0.f, 0.f);
  } else if (EFFECT == MRR_SSM) {
    return make_float3(ssm_at<SMT>(p, in.depth, (const SMT*)in.smap, x, y), 0.f, 0.f);
  } else {
    return ssgi_at<NT>(p, in.depth, (const NT*)in.normal, in.color, x, y);
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

template <int EFFECT, typename NT, typename SMT>
__global__ void __launch_bounds__(SHADE_THREADS) shade_levels_kernel(ShadeParams p, FrameIn in, ShadeLevels lv,
                                                                     int half_store) {
  uint32_t pre[MRR_MAX_LEVELS + 1];
  pre[0] = 0;
  for (int k = 0; k < lv.nlev; ++k)
    pre[k + 1] = pre[k] + min(__ldg(lv.counts + lv.level[k]), (uint32_t)lv.Wi[k] * (uint32_t)lv.Hi[k]);
  const uint32_t total = pre[lv.nlev];
  const int W = p.v.W, H = p.v.H;
  for (uint32_t g = blockIdx.x * SHADE_THREADS + threadIdx.x; g < total; g += gridDim.x * SHADE_THREADS) {
    int k = 0;
    while (g >= pre[k + 1]) ++k;
    const int i = lv.level[k];
    const uint32_t e = __ldg(lv.list[k] + (g - pre[k]));
    const int qx = (int)(e & 0xFFFFu), qy = (int)(e >> 16);
    if (qx >= lv.Wi[k] || qy >= lv.Hi[k]) continue;  // not a texel of this level
    const int o = i == 0 ? 0 : (1 << (i - 1));
    const int x = min((qx << i) + o, W - 1), y = min((qy << i) + o, H - 1);
    const float3 v = effect_at<EFFECT, NT, SMT>(p, in, x, y);
    store_value<EFFECT>(lv.c[k], (size_t)qy * lv.Wi[k] + qx, v, half_store != 0);
  }
}

template <int EFFECT, typename NT, typename SMT>
__global__ void __launch_bounds__(256) shade_full_kernel(ShadeParams p, FrameIn in, float* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.v.W || y >= p.v.H) return;
  const float3 v = effect_at<EFFECT, NT, SMT>(p, in, x, y);
  store_value<EFFECT>(out, (size_t)y * p.v.W + x, v, false);
}

template <int EFFECT, typename NT, typename SMT>
void launch_levels_t(const ShadeParams& p, const FrameIn& in, const ShadeLevels& lv, int half_store, int grid,
                     cudaStream_t s) {
  shade_levels_kernel<EFFECT, NT, SMT><<<grid, SHADE_THREADS, 0, s>>>(p, in, lv, half_store);
}

template <int EFFECT, typename NT, typename SMT>
void launch_full_t(const ShadeParams& p, const FrameIn& in, float* out, cudaStream_t s) {
  dim3 block(32, 8), grid((p.v.W + 31) / 32, (p.v.H + 7) / 8);
  shade_full_kernel<EFFECT, NT, SMT><<<grid, block, 0, s>>>(p, in, out);
}

}  // namespace

std::atomic<uint64_t>& launch_counter() {
  static std::atomic<uint64_t> n{0};
  return n;
}

int shade_grid_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shade_levels_kernel<MRR_SSAO, float4, float>,
                                                  SHADE_THREADS, 0);
    if (sms <= 0) sms = 1;
    if (per_sm <= 0) per_sm = 1;
    blocks = sms * per_sm;
  }
  return blocks;
}

cudaError_t launch_shade_levels(const ShadeParams& p, const FrameIn& in, int precision, const ShadeLevels& lv,
                                int grid, cudaStream_t s) {
  const bool h = precision == MRR_FP16;
  switch (p.effect) {
    case MRR_SSAO:
      if (h) launch_levels_t<MRR_SSAO, half4, __half>(p, in, lv, 1, grid, s);
      else launch_levels_t<MRR_SSAO, float4, float>(p, in, lv, 0, grid, s);
      break;
    case MRR_SSM:
      if (h) launch_levels_t<MRR_SSM, half4, __half>(p, in, lv, 1, grid, s);
      else launch_levels_t<MRR_SSM, float4, float>(p, in, lv, 0, grid, s);
      break;
    default:
      if (h) launch_levels_t<MRR_SSGI, half4, __half>(p, in, lv, 1, grid, s);
      else launch_levels_t<MRR_SSGI, float4, float>(p, in, lv, 0, grid, s);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_shade_full(const ShadeParams& p, const FrameIn& in, int precision, float* out, cudaStream_t s) {
  const bool h = precision == MRR_FP16;
  switch (p.effect) {
    case MRR_SSAO:
      if (h) launch_full_t<MRR_SSAO, half4, __half>(p, in, out, s);
      else launch_full_t<MRR_SSAO, float4, float>(p, in, out, s);
      break;
    case MRR_SSM:
      if (h) launch_full_t<MRR_SSM, half4, __half>(p, in, out, s);
      else launch_full_t<MRR_SSM, float4, float>(p, in, out, s);
      break;
    default:
      if (h) launch_full_t<MRR_SSGI, half4, __half>(p, in, out, s);
      else launch_full_t<MRR_SSGI, float4, float>(p, in, out, s);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
