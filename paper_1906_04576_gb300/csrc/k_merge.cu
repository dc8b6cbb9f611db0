// k_merge.cu -- upsampling and blending of the sub-images (Sec. 4.2, Eq. (1)).
//
// A CTA owns a 32x32 tile of full-resolution pixels, 4 per lane (rows ty, ty+8, ...,
// a warp row is 32 consecutive pixels).  Level texel q sits at full-resolution position
// 2^i q + o_i, so pixel p reads level coordinate u = (p - o_i) / 2^i, whose floor and
// fraction are exactly (p - o_i) >> i and ((p - o_i) & (2^i - 1)) * 2^-i; the taps
// floor(u), floor(u)+1 are clamped to the level.  For every level above 0 the CTA
// stages the (clamped) taps its tile can touch -- a_i, S_i, c_i for at most
// (32/2^i + 2)^2 texels -- in shared memory once, and skips the level for the whole
// tile when none of those texels is rendered (then a_i = 0 there, so alpha = 0).
// Level 0 (one tap, weight 1) is read straight from global memory, c only where
// alpha > 0.  Per pixel, from the coarsest level down: a_i is interpolated plainly,
// c_i over rendered taps with renormalised weights, alpha = min(w_i a_i, 1) and
// c' = c_i alpha + c' (1 - alpha).  Taps of weight exactly 0 are not read (they would
// add +0), and the renormalising division is skipped when the weight sum is exactly 1.
#include "mrr_internal.cuh"

namespace mrr {

namespace {

constexpr int MT = 32;                  // tile side (pixels)
constexpr int FP = MT / 2 + 2;          // largest footprint side (level 1): 18

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

struct LevelTile {
  float a[FP * FP];
  float c[FP * FP][3];
  uint8_t s[FP * FP];
};

struct MergeSmem {
  LevelTile lt[MRR_MAX_LEVELS - 1];   // levels 1..3
  int org_x[MRR_MAX_LEVELS], org_y[MRR_MAX_LEVELS], side[MRR_MAX_LEVELS];
  int any[MRR_MAX_LEVELS];
};

// Eq. (1) step for one level from staged taps.
template <int C>
__device__ __forceinline__ void blend_staged(const MergeParams& p, const LevelTile& t, int i, int ox, int oy,
                                             int side, int x, int y, bool first, float& c0, float& c1,
                                             float& c2) {
  const int o = 1 << (i - 1), mask = (1 << i) - 1;
  const float inv = __int_as_float((127 - i) << 23);  // 2^-i
  const int tx = x - o, ty = y - o;
  const float fx = (float)(tx & mask) * inv, fy = (float)(ty & mask) * inv;
  const int lx = (tx >> i) - ox, ly = (ty >> i) - oy;
  const int base = ly * side + lx;
  const int idx[4] = {base, base + 1, base + side, base + side + 1};
  const float w[4] = {(1.0f - fx) * (1.0f - fy), fx * (1.0f - fy), (1.0f - fx) * fy, fx * fy};
  float ahat = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (w[k] != 0.0f) ahat = ahat + w[k] * t.a[idx[k]];
  const float wa = p.weight[i] * ahat;
  const float alpha = (1.0f < wa) ? 1.0f : wa;
  if (!first && !(alpha > 0.0f)) return;
  float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (w[k] == 0.0f || !t.s[idx[k]]) continue;
    n0 = n0 + w[k] * t.c[idx[k]][0];
    if (C == 4) {
      n1 = n1 + w[k] * t.c[idx[k]][1];
      n2 = n2 + w[k] * t.c[idx[k]][2];
    }
    den = den + w[k];
  }
  if (den != 1.0f) {
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
  __shared__ MergeSmem sm;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int X0 = blockIdx.x * MT, Y0 = blockIdx.y * MT;
  // stage the footprints of levels 1..L-1
  for (int i = 1; i < p.L; ++i) {
    if (!p.enabled[i]) continue;
    const int o = 1 << (i - 1);
    const int fx0 = (X0 - o) >> i, fy0 = (Y0 - o) >> i;
    const int side = ((X0 + MT - 1 - o) >> i) - fx0 + 2;
    const int rows = ((Y0 + MT - 1 - o) >> i) - fy0 + 2;
    if (threadIdx.x == 0) {
      sm.org_x[i] = fx0;
      sm.org_y[i] = fy0;
      sm.side[i] = side;
    }
    LevelTile& t = sm.lt[i - 1];
    int any = 0;
    const int Wi = p.Wi[i], Hi = p.Hi[i];
    for (int k = threadIdx.x; k < side * rows; k += 256) {
      const int ly = k / side, lx = k - ly * side;
      const int qx = min(max(fx0 + lx, 0), Wi - 1), qy = min(max(fy0 + ly, 0), Hi - 1);
      const size_t q = (size_t)qy * Wi + qx;
      const uint8_t s = __ldg(p.stencil[i] + q);
      t.s[k] = s;
      t.a[k] = __ldg(p.alpha[i] + q);
      if (s) {
        const float3 v = load_c<CT>(p.c[i], q, C);
        t.c[k][0] = v.x;
        t.c[k][1] = v.y;
        t.c[k][2] = v.z;
      }
      any |= s;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) sm.any[i] = any;
  }
  __syncthreads();
  const int W = p.W, H = p.H;
  const int x = X0 + tx;
  for (int r = ty; r < MT; r += 8) {
    const int y = Y0 + r;
    if (x >= W || y >= H) continue;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    bool first = true;
    for (int i = p.L - 1; i >= 1; --i) {
      if (!p.enabled[i] || (!first && !sm.any[i])) continue;
      blend_staged<C>(p, sm.lt[i - 1], i, sm.org_x[i], sm.org_y[i], sm.side[i], x, y, first, c0, c1, c2);
      first = false;
    }
    if (p.enabled[0]) {
      const size_t q = (size_t)y * W + x;
      const float a0 = __ldg(p.alpha[0] + q);
      const float ahat = 0.0f + 1.0f * a0;
      const float wa = p.weight[0] * ahat;
      const float alpha = (1.0f < wa) ? 1.0f : wa;
      if (first || alpha > 0.0f) {
        float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f;
        if (__ldg(p.stencil[0] + q)) {
          const float3 v = load_c<CT>(p.c[0], q, C);
          n0 = v.x;
          n1 = v.y;
          n2 = v.z;
          den = 1.0f;
        } else {
          n0 = n0 / den;  // no rendered tap: 0/0, as the definition gives
          n1 = n1 / den;
          n2 = n2 / den;
        }
        if (first) {
          c0 = n0;
          c1 = n1;
          c2 = n2;
        } else {
          const float om = 1.0f - alpha;
          c0 = n0 * alpha + c0 * om;
          if (C == 4) {
            c1 = n1 * alpha + c1 * om;
            c2 = n2 * alpha + c2 * om;
          }
        }
      }
    }
    const size_t o = (size_t)y * W + x;
    if (C == 4)
      reinterpret_cast<float4*>(out)[o] = make_float4(c0, c1, c2, 0.0f);
    else
      out[o] = c0;
  }
}

}  // namespace

cudaError_t launch_merge(const MergeParams& p, float* out, cudaStream_t s) {
  dim3 grid((p.W + MT - 1) / MT, (p.H + MT - 1) / MT);
  if (p.C == 4) {
    if (p.half_store) merge_kernel<__half, 4><<<grid, 256, 0, s>>>(p, out);
    else merge_kernel<float, 4><<<grid, 256, 0, s>>>(p, out);
  } else {
    if (p.half_store) merge_kernel<__half, 1><<<grid, 256, 0, s>>>(p, out);
    else merge_kernel<float, 1><<<grid, 256, 0, s>>>(p, out);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
