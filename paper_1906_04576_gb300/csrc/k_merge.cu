// k_merge.cu -- upsampling and blending of the sub-images (Sec. 4.2, Eq. (1)).
//
// One thread per full-resolution pixel, 64x4 tiles (a warp covers 32 consecutive pixels
// of a row, so the level reads of neighbouring lanes share cache lines).  From the
// coarsest enabled level to the finest: level texel q sits at full-resolution position
// 2^i q + o_i, pixel p reads level coordinate u = (p - o_i) / 2^i (exact in binary
// floating point), the four taps floor(u), floor(u)+1 are clamped to the level; a_i is
// interpolated plainly, c_i over rendered taps only with renormalised weights, and
// alpha = min(w_i a_i, 1), c' = c_i alpha + c' (1 - alpha).  Taps whose bilinear weight
// is exactly zero are not read: they would add exactly +0 to each sum.
#include "mrr_internal.cuh"

namespace mrr {

namespace {

template <typename CT> __device__ __forceinline__ float3 load_c(const void* c, size_t i, int C);

template <> __device__ __forceinline__ float3 load_c<float>(const void* c, size_t i, int C) {
  if (C == 1) return make_float3(__ldg(reinterpret_cast<const float*>(c) + i), 0.f, 0.f);
  const float4 v = __ldg(reinterpret_cast<const float4*>(c) + i);
  return make_float3(v.x, v.y, v.z);
}

template <> __device__ __forceinline__ float3 load_c<__half>(const void* c, size_t i, int C) {
  if (C == 1) return make_float3(__half2float(__ldg(reinterpret_cast<const __half*>(c) + i)), 0.f, 0.f);
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(c) + i);
  const __half2 xy = *reinterpret_cast<const __half2*>(&raw.x);
  const __half2 zw = *reinterpret_cast<const __half2*>(&raw.y);
  return make_float3(__low2float(xy), __high2float(xy), __low2float(zw));
}

// Blend of one level into the composite c (Eq. (1)); `first` = the coarsest level,
// which initialises c.  Level coordinate of pixel x: u = (x - o_i) / 2^i, whose floor and
// fraction are (x - o_i) >> i and ((x - o_i) & (2^i - 1)) * 2^-i exactly.
template <typename CT, int C>
__device__ __forceinline__ void blend_level(const MergeParams& p, int i, int x, int y, bool first, float& c0,
                                            float& c1, float& c2) {
  const int Wi = p.Wi[i], Hi = p.Hi[i];
  int tx = x, ty = y, x0 = x, y0 = y;
  float fx = 0.0f, fy = 0.0f;
  if (i > 0) {
    const int o = 1 << (i - 1), mask = (1 << i) - 1;
    const float inv = __int_as_float((127 - i) << 23);  // 2^-i
    tx = x - o;
    ty = y - o;
    x0 = tx >> i;
    y0 = ty >> i;
    fx = (float)(tx & mask) * inv;
    fy = (float)(ty & mask) * inv;
  }
  const int xa = min(max(x0, 0), Wi - 1), xb = min(max(x0 + 1, 0), Wi - 1);
  const int ya = min(max(y0, 0), Hi - 1), yb = min(max(y0 + 1, 0), Hi - 1);
  const float w[4] = {(1.0f - fx) * (1.0f - fy), fx * (1.0f - fy), (1.0f - fx) * fy, fx * fy};
  const int idx[4] = {ya * Wi + xa, ya * Wi + xb, yb * Wi + xa, yb * Wi + xb};
  float ahat = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (w[k] != 0.0f) ahat = ahat + w[k] * __ldg(p.alpha[i] + idx[k]);
  const float wa = p.weight[i] * ahat;
  const float alpha = (1.0f < wa) ? 1.0f : wa;
  if (!first && !(alpha > 0.0f)) return;
  float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (w[k] == 0.0f || !__ldg(p.stencil[i] + idx[k])) continue;
    const float3 v = load_c<CT>(p.c[i], idx[k], C);
    n0 = n0 + w[k] * v.x;
    if (C == 4) {
      n1 = n1 + w[k] * v.y;
      n2 = n2 + w[k] * v.z;
    }
    den = den + w[k];
  }
  if (den != 1.0f) {  // x / 1 is x: the division only matters when a tap was dropped
    n0 = n0 / den;
    if (C == 4) {
      n1 = n1 / den;
      n2 = n2 / den;
    }
  }
  if (first) {
    c0 = n0;
    c1 = n1;
    c2 = n2;
    return;
  }
  const float om = 1.0f - alpha;
  c0 = n0 * alpha + c0 * om;
  if (C == 4) {
    c1 = n1 * alpha + c1 * om;
    c2 = n2 * alpha + c2 * om;
  }
}

template <typename CT, int C>
__global__ void __launch_bounds__(256) merge_kernel(MergeParams p, float* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.W || y >= p.H) return;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f;
  blend_level<CT, C>(p, p.L - 1, x, y, true, c0, c1, c2);
  for (int i = p.L - 2; i >= 0; --i)
    if (p.enabled[i]) blend_level<CT, C>(p, i, x, y, false, c0, c1, c2);
  const size_t o = (size_t)y * p.W + x;
  if (C == 4)
    reinterpret_cast<float4*>(out)[o] = make_float4(c0, c1, c2, 0.0f);
  else
    out[o] = c0;
}

}  // namespace

cudaError_t launch_merge(const MergeParams& p, float* out, cudaStream_t s) {
  dim3 block(64, 4), grid((p.W + 63) / 64, (p.H + 3) / 4);
  if (p.C == 4) {
    if (p.half_store) merge_kernel<__half, 4><<<grid, block, 0, s>>>(p, out);
    else merge_kernel<float, 4><<<grid, block, 0, s>>>(p, out);
  } else {
    if (p.half_store) merge_kernel<__half, 1><<<grid, block, 0, s>>>(p, out);
    else merge_kernel<float, 1><<<grid, block, 0, s>>>(p, out);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
