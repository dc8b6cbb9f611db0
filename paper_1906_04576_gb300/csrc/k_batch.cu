// k_batch.cu -- one persistent launch that shades the work lists of several frames at
// once (frames of different sizes and different effects), pulling chunks of work from
// a global tile queue.
//
// The queue is implicit: the concatenation, in (item, level) order, of every item's
// work lists, whose lengths are read on the device.  A CTA takes the next chunk of
// `chunk` entries with one atomicAdd on the queue head (reset to 0 by the caller before
// the launch), so expensive items (SSGI) and cheap ones (SSAO) balance across SMs
// without any host synchronisation.  Every entry is shaded with exactly the effect
// function the single-frame kernels use, so a batched frame equals the same frame
// rendered alone, bit for bit.
#include "mrr_internal.cuh"
#include "shade_common.cuh"

namespace mrr {

namespace {

constexpr int BATCH_THREADS = 256;

template <typename NT, typename SMT>
__device__ __forceinline__ float3 batch_effect(const ShadeParams& p, const FrameIn& in, int x, int y) {
  if (p.effect == MRR_SSAO) {
    return make_float3(ssao_at<NT, 1>(p, in.depth, (const NT*)in.normal, x, y, true), 0.f, 0.f);
  } else if (p.effect == MRR_SSM) {
    return make_float3(ssm_at<SMT>(p, in.depth, (const SMT*)in.smap, x, y), 0.f, 0.f);
  }
  return ssgi_at<NT>(p, in.depth, (const NT*)in.normal, in.color, x, y);
}

__device__ __forceinline__ void batch_store(void* c, size_t i, float3 v, int effect, int half_store) {
  if (effect == MRR_SSGI) {
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
  } else if (half_store) {
    reinterpret_cast<__half*>(c)[i] = __float2half_rn(v.x);
  } else {
    reinterpret_cast<float*>(c)[i] = v.x;
  }
}

// All three effects share one kernel, so its registers are those of the largest (SSGI).
// The kernel waits mostly on its gathers; capped at 64 registers (4 CTAs, 32 warps per SM,
// a 16-byte spill) it shades the batched SSGI + SSAO 4K frames 3 % faster than at its
// unconstrained 71 (3 CTAs); at 48 registers the spills cost more than the warps gain.
__global__ void __launch_bounds__(BATCH_THREADS, 4) shade_batch_kernel(const BatchItem* __restrict__ items, int nitems,
                                                                    uint32_t* queue_head, int chunk) {
  // segment s = (item, level slot); prefix of the segment lengths
  __shared__ uint32_t s_pre[MAX_BATCH * MRR_MAX_LEVELS + 1];
  __shared__ uint32_t s_take;
  const int nseg = nitems * MRR_MAX_LEVELS;
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    s_pre[0] = 0;
    for (int s = 0; s < nseg; ++s) {
      const BatchItem& it = items[s / MRR_MAX_LEVELS];
      const int k = s % MRR_MAX_LEVELS;
      uint32_t n = 0;
      if (k < it.lv.nlev)
        n = min(__ldg(it.lv.counts + it.lv.level[k]), (uint32_t)it.lv.Wi[k] * (uint32_t)it.lv.Hi[k]);
      acc += n;
      s_pre[s + 1] = acc;
    }
  }
  __syncthreads();
  const uint32_t total = s_pre[nseg];
  for (;;) {
    if (threadIdx.x == 0) s_take = atomicAdd(queue_head, 1u);
    __syncthreads();
    const uint32_t start = s_take * (uint32_t)chunk;
    __syncthreads();  // s_take is reused by the next iteration
    if (start >= total) break;
    const uint32_t end = min(start + (uint32_t)chunk, total);
    for (uint32_t g = start + threadIdx.x; g < end; g += BATCH_THREADS) {
      int s = 0;
      while (g >= s_pre[s + 1]) ++s;
      const BatchItem& it = items[s / MRR_MAX_LEVELS];
      const int k = s % MRR_MAX_LEVELS;
      const int i = it.lv.level[k];
      const uint32_t e = __ldg(it.lv.list[k] + (g - s_pre[s]));
      const int qx = (int)(e & 0xFFFFu), qy = (int)(e >> 16);
      if (qx >= it.lv.Wi[k] || qy >= it.lv.Hi[k]) continue;  // not a texel of the level
      const int o = i == 0 ? 0 : (1 << (i - 1));
      const int x = min((qx << i) + o, it.p.v.W - 1), y = min((qy << i) + o, it.p.v.H - 1);
      float3 v;
      if (it.precision == MRR_FP16) v = batch_effect<half4, float>(it.p, it.in, x, y);
      else v = batch_effect<float4, float>(it.p, it.in, x, y);
      const size_t at = ((it.lv.compact >> k) & 1) ? (size_t)(g - s_pre[s]) : (size_t)qy * it.lv.Wi[k] + qx;
      batch_store(it.lv.c[k], at, v, it.p.effect, it.precision == MRR_FP16);
    }
  }
}

}  // namespace

int batch_grid_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shade_batch_kernel, BATCH_THREADS, 0);
    blocks = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  }
  return blocks;
}

cudaError_t launch_shade_batch(const BatchItem* items_dev, int nitems, uint32_t* queue_head, int chunk, int grid,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(queue_head, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  shade_batch_kernel<<<grid, BATCH_THREADS, 0, s>>>(items_dev, nitems, queue_head, chunk);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
