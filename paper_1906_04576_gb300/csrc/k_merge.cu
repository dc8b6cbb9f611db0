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
// c' = c_i alpha + c' (1 - alpha).  A tap of weight 0 adds +0 either way, and the
// renormalising division is skipped when the weight sum is exactly 1 (x / 1 = x).
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

constexpr int ROWS = MT / 8;  // pixel rows per lane

// Stage the (clamped) taps of level I that the tile can touch; returns via sm.any[I]
// whether any of them is rendered.
template <typename CT, int C, int I>
__device__ __forceinline__ void stage_level(const MergeParams& p, MergeSmem& sm, int X0, int Y0) {
  constexpr int o = 1 << (I - 1);
  // X0 is a multiple of MT, so the footprint is (MT >> I) + 2 texels on each side
  constexpr int side = (MT >> I) + 2, rows = side;
  const int fx0 = (X0 - o) >> I, fy0 = (Y0 - o) >> I;
  LevelTile& t = sm.lt[I - 1];
  const int Wi = p.Wi[I], Hi = p.Hi[I];
  int any = 0;
  for (int k = threadIdx.x; k < side * rows; k += 256) {
    const int ly = k / side, lx = k - ly * side;
    const int qx = min(max(fx0 + lx, 0), Wi - 1), qy = min(max(fy0 + ly, 0), Hi - 1);
    const size_t q = (size_t)qy * Wi + qx;
    const uint8_t st = __ldg(p.stencil[I] + q);
    t.s[k] = st;
    t.a[k] = __ldg(p.alpha[I] + q);
    if (st) {
      const float3 v = load_c<CT>(p.c[I], q, C);
      t.c[k][0] = v.x;
      t.c[k][1] = v.y;
      t.c[k][2] = v.z;
    }
    any |= st;
  }
  if (threadIdx.x == 0) {
    sm.org_x[I] = fx0;
    sm.org_y[I] = fy0;
    sm.side[I] = side;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) sm.any[I] = any;
}

// Eq. (1) for level I (compile-time) on the lane's ROWS pixels of column x.
template <int C, int I>
__device__ __forceinline__ void blend_rows(const MergeParams& p, const MergeSmem& sm, int x, int Y0, int ty,
                                           bool first, float (&c)[ROWS][3]) {
  constexpr int o = 1 << (I - 1), mask = (1 << I) - 1;
  const float inv = __int_as_float((127 - I) << 23);  // 2^-I
  const LevelTile& t = sm.lt[I - 1];
  constexpr int side = (MT >> I) + 2;
  const int tx = x - o;
  const float fx = (float)(tx & mask) * inv;
  const float gx = 1.0f - fx;
  const int lx = (tx >> I) - sm.org_x[I];
  const float weight = p.weight[I];
#pragma unroll
  for (int rr = 0; rr < ROWS; ++rr) {
    const int y = Y0 + ty + 8 * rr;
    const int tyy = y - o;
    const float fy = (float)(tyy & mask) * inv;
    const float gy = 1.0f - fy;
    const int base = ((tyy >> I) - sm.org_y[I]) * side + lx;
    const int idx[4] = {base, base + 1, base + side, base + side + 1};
    const float w[4] = {gx * gy, fx * gy, gx * fy, fx * fy};
    // every tap is added (a weight of 0 adds +0); unrendered taps add +0 through a select
    float ahat = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) ahat = ahat + w[k] * t.a[idx[k]];
    const float wa = weight * ahat;
    const float alpha = (1.0f < wa) ? 1.0f : wa;
    if (!first && !(alpha > 0.0f)) continue;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool on = t.s[idx[k]] != 0;
      n0 = n0 + (on ? w[k] * t.c[idx[k]][0] : 0.0f);
      if (C == 4) {
        n1 = n1 + (on ? w[k] * t.c[idx[k]][1] : 0.0f);
        n2 = n2 + (on ? w[k] * t.c[idx[k]][2] : 0.0f);
      }
      den = den + (on ? w[k] : 0.0f);
    }
    if (den != 1.0f) {
      n0 = n0 / den;
      if (C == 4) {
        n1 = n1 / den;
        n2 = n2 / den;
      }
    }
    if (first) {
      c[rr][0] = n0;
      c[rr][1] = n1;
      c[rr][2] = n2;
    } else {
      const float om = 1.0f - alpha;
      c[rr][0] = n0 * alpha + c[rr][0] * om;
      if (C == 4) {
        c[rr][1] = n1 * alpha + c[rr][1] * om;
        c[rr][2] = n2 * alpha + c[rr][2] * om;
      }
    }
  }
}

template <typename CT, int C, int L>
__global__ void __launch_bounds__(256) merge_kernel(MergeParams p, float* __restrict__ out) {
  __shared__ MergeSmem sm;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int X0 = blockIdx.x * MT, Y0 = blockIdx.y * MT;
  if (L > 1 && p.enabled[1]) stage_level<CT, C, 1>(p, sm, X0, Y0);
  if (L > 2 && p.enabled[2]) stage_level<CT, C, (L > 2 ? 2 : 1)>(p, sm, X0, Y0);
  if (L > 3) stage_level<CT, C, (L > 3 ? 3 : 1)>(p, sm, X0, Y0);
  __syncthreads();
  const int W = p.W, H = p.H;
  const int x = X0 + tx;
  if (x >= W) return;
  float c[ROWS][3] = {};
  // coarsest level first, then the finer enabled levels that the tile touches
  bool first = true;
  if (L == 4) {
    blend_rows<C, (L == 4 ? 3 : 1)>(p, sm, x, Y0, ty, true, c);
    first = false;
  }
  if (L >= 3 && p.enabled[2] && (first || sm.any[2])) {
    blend_rows<C, (L >= 3 ? 2 : 1)>(p, sm, x, Y0, ty, first, c);
    first = false;
  }
  if (L >= 2 && p.enabled[1] && (first || sm.any[1])) {
    blend_rows<C, 1>(p, sm, x, Y0, ty, first, c);
    first = false;
  }
  if (p.enabled[0]) {
#pragma unroll
    for (int rr = 0; rr < ROWS; ++rr) {
      const int y = Y0 + ty + 8 * rr;
      if (y >= H) break;
      const size_t q = (size_t)y * W + x;
      const float a0 = __ldg(p.alpha[0] + q);
      const float ahat = 0.0f + 1.0f * a0;
      const float wa = p.weight[0] * ahat;
      const float alpha = (1.0f < wa) ? 1.0f : wa;
      if (!first && !(alpha > 0.0f)) continue;
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
        c[rr][0] = n0;
        c[rr][1] = n1;
        c[rr][2] = n2;
      } else {
        const float om = 1.0f - alpha;
        c[rr][0] = n0 * alpha + c[rr][0] * om;
        if (C == 4) {
          c[rr][1] = n1 * alpha + c[rr][1] * om;
          c[rr][2] = n2 * alpha + c[rr][2] * om;
        }
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < ROWS; ++rr) {
    const int y = Y0 + ty + 8 * rr;
    if (y >= H) break;
    const size_t o = (size_t)y * W + x;
    if (C == 4)
      reinterpret_cast<float4*>(out)[o] = make_float4(c[rr][0], c[rr][1], c[rr][2], 0.0f);
    else
      out[o] = c[rr][0];
  }
}

template <typename CT, int C>
void launch_merge_t(const MergeParams& p, float* out, cudaStream_t s) {
  dim3 grid((p.W + MT - 1) / MT, (p.H + MT - 1) / MT);
  switch (p.L) {
    case 1: merge_kernel<CT, C, 1><<<grid, 256, 0, s>>>(p, out); break;
    case 2: merge_kernel<CT, C, 2><<<grid, 256, 0, s>>>(p, out); break;
    case 3: merge_kernel<CT, C, 3><<<grid, 256, 0, s>>>(p, out); break;
    default: merge_kernel<CT, C, 4><<<grid, 256, 0, s>>>(p, out); break;
  }
}

}  // namespace

cudaError_t launch_merge(const MergeParams& p, float* out, cudaStream_t s) {
  if (p.C == 4) {
    if (p.half_store) launch_merge_t<__half, 4>(p, out, s);
    else launch_merge_t<float, 4>(p, out, s);
  } else {
    if (p.half_store) launch_merge_t<__half, 1>(p, out, s);
    else launch_merge_t<float, 1>(p, out, s);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
