// k_masks.cu -- the per-level masks of Sec. 3.1 / Table 1, the stencil of Sec. 4.1 and
// the dense work lists that replace the stencil test on the GPU.
//
// mask_level_kernel: one CTA per 32x16 tile of level texels.  It stages the downsampled
//   edge image D_i (block maximum of the edge image) for the tile plus an R_i halo in
//   shared memory, blurs it horizontally into a second shared buffer and vertically
//   into a_i, sets S_i = [a_i > 0] and ORs in the set texels of the previous enabled
//   finer level inside the texel's block (inclusive nesting, Fig. 2/3).
// compact_count_kernel / compact_scatter_kernel: deterministic stream compaction of
//   every level's stencil into a row-major list of (y << 16) | x.  Pass 1 counts the set
//   texels of each 4096-texel chunk; pass 2 gives each chunk its exclusive prefix (a
//   block reduction over the preceding chunk counts of its level) and scatters with a
//   warp ballot + popc per 256-texel round, so list order = index order and no warp of
//   the shading kernel idles on an unmasked texel.
// label_kernel: the owning level of each full-resolution pixel.
#include "mrr_internal.cuh"

namespace mrr {

namespace {

constexpr int MTX = 32, MTY = 16, MAXR = 6;

__global__ void __launch_bounds__(256) mask_level_kernel(MaskLevel m, const uint8_t* __restrict__ E, int W, int H) {
  __shared__ float sD[MTY + 2 * MAXR][MTX + 2 * MAXR];
  __shared__ float sh[MTY + 2 * MAXR][MTX];
  const int tid = threadIdx.x;
  const int tx0 = blockIdx.x * MTX, ty0 = blockIdx.y * MTY;
  const int Wi = m.Wi, Hi = m.Hi;
  if (m.mode != 0) {
    const float av = m.mode == 1 ? 1.0f : 0.0f;
    const uint8_t sv = m.mode == 1 ? 1 : 0;
    for (int k = tid; k < MTX * MTY; k += blockDim.x) {
      const int qx = tx0 + (k % MTX), qy = ty0 + (k / MTX);
      if (qx < Wi && qy < Hi) {
        m.alpha[(size_t)qy * Wi + qx] = av;
        m.stencil[(size_t)qy * Wi + qx] = sv;
      }
    }
    return;
  }
  const int R = m.R;
  const int DX = MTX + 2 * R, DY = MTY + 2 * R;
  const int bs = 1 << m.level;
  for (int k = tid; k < DX * DY; k += blockDim.x) {
    const int ly = k / DX, lx = k - ly * DX;
    const int qx = tx0 - R + lx, qy = ty0 - R + ly;
    float v = 0.0f;
    if (qx >= 0 && qx < Wi && qy >= 0 && qy < Hi) {
      const int xa = qx * bs, ya = qy * bs;
      const int xb = min(xa + bs, W), yb = min(ya + bs, H);
      uint8_t mx = 0;
      for (int y = ya; y < yb; ++y)
        for (int x = xa; x < xb; ++x) mx |= __ldg(E + (size_t)y * W + x);
      v = mx ? 1.0f : 0.0f;
    }
    sD[ly][lx] = v;
  }
  __syncthreads();
  for (int k = tid; k < DY * MTX; k += blockDim.x) {
    const int ly = k / MTX, lx = k - ly * MTX;
    float s = 0.0f;
    for (int t = 0; t <= 2 * R; ++t) s = s + m.g[t] * sD[ly][lx + t];
    sh[ly][lx] = s;
  }
  __syncthreads();
  for (int k = tid; k < MTX * MTY; k += blockDim.x) {
    const int ly = k / MTX, lx = k - ly * MTX;
    const int qx = tx0 + lx, qy = ty0 + ly;
    if (qx >= Wi || qy >= Hi) continue;
    float s = 0.0f;
    for (int t = 0; t <= 2 * R; ++t) s = s + m.g[t] * sh[ly + t][lx];
    uint8_t st = s > 0.0f ? 1 : 0;
    if (!st && m.prev) {
      const int f = 1 << m.prev_shift;
      const int xa = qx * f, ya = qy * f;
      const int xb = min(xa + f, m.prev_W), yb = min(ya + f, m.prev_H);
      for (int y = ya; y < yb && !st; ++y)
        for (int x = xa; x < xb; ++x) st |= __ldg(m.prev + (size_t)y * m.prev_W + x);
    }
    m.alpha[(size_t)qy * Wi + qx] = s;
    m.stencil[(size_t)qy * Wi + qx] = st;
  }
}

// Which (slot, chunk-in-level) does this block own?
__device__ __forceinline__ int slot_of(const CompactParams& p, int b) {
  int l = 0;
  while (l + 1 < p.nlev && b >= p.chunk_begin[l + 1]) ++l;
  return l;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  uint32_t t = 0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < COMPACT_THREADS / 32; ++w) t += red[w];
    red[COMPACT_THREADS / 32] = t;
  }
  __syncthreads();
  t = red[COMPACT_THREADS / 32];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(COMPACT_THREADS) compact_count_kernel(CompactParams p) {
  __shared__ uint32_t red[COMPACT_THREADS / 32 + 1];
  const int l = slot_of(p, blockIdx.x);
  const int c = blockIdx.x - p.chunk_begin[l];
  const size_t n = (size_t)p.Wi[l] * p.Hi[l];
  const uint8_t* S = p.stencil[l];
  const size_t base = (size_t)c * COMPACT_CHUNK + (size_t)threadIdx.x * (COMPACT_CHUNK / COMPACT_THREADS);
  uint32_t cnt = 0;
  if (base + 16 <= n && ((reinterpret_cast<uintptr_t>(S + base) & 15) == 0)) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(S + base));
    cnt = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);  // bytes are 0 or 1
  } else {
    for (size_t k = base; k < base + 16 && k < n; ++k) cnt += S[k] ? 1u : 0u;
  }
  const uint32_t tot = block_sum(cnt, red);
  if (threadIdx.x == 0) p.chunk_counts[blockIdx.x] = tot;
  if (blockIdx.x == 0 && threadIdx.x < MRR_MAX_LEVELS && ((p.zero_mask >> threadIdx.x) & 1))
    p.counts[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(COMPACT_THREADS) compact_scatter_kernel(CompactParams p) {
  __shared__ uint32_t red[COMPACT_THREADS / 32 + 1];
  __shared__ uint32_t wsum[COMPACT_THREADS / 32];
  const int l = slot_of(p, blockIdx.x);
  const int c0 = p.chunk_begin[l];
  const int c = blockIdx.x - c0;
  // exclusive prefix of this chunk within its level
  uint32_t part = 0;
  for (int k = c0 + threadIdx.x; k < (int)blockIdx.x; k += COMPACT_THREADS) part += p.chunk_counts[k];
  uint32_t offset = block_sum(part, red);
  const int Wi = p.Wi[l];
  const size_t n = (size_t)Wi * p.Hi[l];
  const uint8_t* S = p.stencil[l];
  uint32_t* list = p.list[l];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t base = (size_t)c * COMPACT_CHUNK;
  for (int round = 0; round < COMPACT_CHUNK / COMPACT_THREADS; ++round) {
    const size_t idx = base + (size_t)round * COMPACT_THREADS + threadIdx.x;
    const bool set = idx < n && S[idx] != 0;
    const uint32_t bal = __ballot_sync(0xffffffffu, set);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < COMPACT_THREADS / 32; ++w) {
      const uint32_t s = wsum[w];
      before += (w < warp) ? s : 0u;
      total += s;
    }
    if (set) {
      const uint32_t pos = offset + before + __popc(bal & ((1u << lane) - 1u));
      const uint32_t y = (uint32_t)(idx / Wi), x = (uint32_t)(idx - (size_t)y * Wi);
      list[pos] = (y << 16) | x;
    }
    offset += total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && (int)blockIdx.x == p.chunk_begin[l + 1] - 1) p.counts[p.level_of[l]] = offset;
}

struct LabelParams {
  int nlev;
  int level[MRR_MAX_LEVELS];
  const uint8_t* stencil[MRR_MAX_LEVELS];
  int Wi[MRR_MAX_LEVELS];
};

__global__ void label_kernel(LabelParams lp, uint8_t* __restrict__ label, int W, int H) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  uint8_t lab = 0xFF;
  for (int k = 0; k < lp.nlev; ++k) {
    const int i = lp.level[k];
    if (__ldg(lp.stencil[k] + (size_t)(y >> i) * lp.Wi[k] + (x >> i))) {
      lab = (uint8_t)i;
      break;
    }
  }
  label[(size_t)y * W + x] = lab;
}

}  // namespace

cudaError_t launch_mask_level(const MaskLevel& m, const uint8_t* E, int W, int H, cudaStream_t s) {
  dim3 grid((m.Wi + MTX - 1) / MTX, (m.Hi + MTY - 1) / MTY);
  mask_level_kernel<<<grid, 256, 0, s>>>(m, E, W, H);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_compact(const CompactParams& p, cudaStream_t s) {
  const int nchunks = p.chunk_begin[p.nlev];
  if (nchunks > 0) {
    compact_count_kernel<<<nchunks, COMPACT_THREADS, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    compact_scatter_kernel<<<nchunks, COMPACT_THREADS, 0, s>>>(p);
    count_launches(2);
  }
  return cudaGetLastError();
}

cudaError_t launch_label(uint8_t* label, int W, int H, int nlev, const int* levels, const uint8_t* const* stencil,
                         const int* Wi, cudaStream_t s) {
  LabelParams lp;
  lp.nlev = nlev;
  for (int k = 0; k < nlev; ++k) {
    lp.level[k] = levels[k];
    lp.stencil[k] = stencil[k];
    lp.Wi[k] = Wi[k];
  }
  dim3 block(64, 4), grid((W + 63) / 64, (H + 3) / 4);
  label_kernel<<<grid, block, 0, s>>>(lp, label, W, H);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
