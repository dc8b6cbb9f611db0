// k_merge.cu -- upsampling and blending of the sub-images (Sec. 4.2, Eq. (1)).
//
// A CTA owns a 32x16 tile of full-resolution pixels (128 threads, so that many tiles are
// in flight per SM); warp w owns the 4 consecutive rows 4w .. 4w+3 and lane x the column.  Level texel q sits at full-resolution position
// 2^i q + o_i, so pixel p reads level coordinate u = (p - o_i) / 2^i, whose floor and
// fraction are exactly (p - o_i) >> i and ((p - o_i) & (2^i - 1)) * 2^-i; the taps
// floor(u), floor(u)+1 are clamped to the level.  For every level above 0 the CTA stages
// the (clamped) taps its tile can touch -- (32/2^i + 2) x (16/2^i + 2) texels -- in shared
// memory once: a_i, the stencil as 0/1 and c_i with unrendered texels replaced by 0, so
// that w * c and w * s are exactly the terms a rendered tap adds and +0 otherwise.  The
// 4 rows of a warp touch only 4 / 3 / 2 footprint rows of levels 1 / 2 / 3, which the lane
// reads once into registers.  A level none of whose staged a_i is positive is skipped
// for the tile (alpha = 0 there).  Level 0 (one tap, weight 1) is read from global memory,
// c only where it is blended.  Per pixel, from the coarsest level down: a_i interpolated
// plainly, c_i over rendered taps with renormalised weights, alpha = min(w_i a_i, 1) and
// c' = c_i alpha + c' (1 - alpha); the coarsest level is taken as is.  The renormalising
// division is skipped when the weight sum is exactly 1 (x / 1 = x).
//
// chain_kernel: the step-wise reading of Sec. 3.3 instead -- one launch per step, each
// level's composite computed at its own resolution from the previous one.
// merge_samples_kernel: the blend of sample-count levels (full-resolution sub-images).
// merge_bilateral_kernel: the direct merge with depth-aware (bilateral) taps.
#include "mrr_internal.cuh"

namespace mrr {

namespace {

constexpr int MTHR = 128;               // threads per CTA
constexpr int RPW = 4;                  // consecutive pixel rows per warp
constexpr int MTX = 32;                 // tile width (pixels): a warp row
constexpr int MTY = RPW * (MTHR / 32);  // tile height (pixels)

template <int I> struct Lv {
  static constexpr int side = (MTX >> I) + 2;  // footprint columns of the tile at level I (row stride)
  static constexpr int rows = (MTY >> I) + 2;  // footprint rows
  static constexpr int n = side * rows;
  static constexpr int o = I == 0 ? 0 : (1 << (I - 1));
  static constexpr int mask = (1 << I) - 1;
  // footprint rows that the RPW rows of a warp touch (tap rows included)
  static constexpr int nr = I == 1 ? 4 : (I == 2 ? 3 : 2);
};
// staged entries: level 1, then level 2, then level 3
template <int I> constexpr int lv_off() { return I <= 1 ? 0 : (I == 2 ? Lv<1>::n : Lv<1>::n + Lv<2>::n); }
constexpr int NTAP = Lv<1>::n + Lv<2>::n + Lv<3>::n;
static_assert(MTY % 8 == 0 && MTX % 8 == 0, "tiles cover whole level-3 texels");

template <int C> struct MergeSmem {
  float a[NTAP];
  float s[NTAP];
  float cz[C == 4 ? 3 : 1][NTAP];
  int any[MTHR / 32];
};

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

// One staged footprint entry kk of level I: the clamped texel's stencil, a and c.
template <typename CT, int C, int I>
__device__ __forceinline__ void load_entry(const MergeParams& p, int X0, int Y0, int kk, uint8_t& st, float& av,
                                           float3& cv) {
  constexpr int side = Lv<I>::side;
  const int ly = kk / side, lx = kk - ly * side;
  const int Wi = p.Wi[I], Hi = p.Hi[I];
  // footprint origin: (X0 - o_I) >> I = X0 / 2^I - 1, X0 and Y0 being multiples of 8
  const int qx = min(max((X0 >> I) - 1 + lx, 0), Wi - 1);
  const int qy = min(max((Y0 >> I) - 1 + ly, 0), Hi - 1);
  const size_t q = (size_t)qy * Wi + qx;
  st = __ldg(p.stencil[I] + q);
  av = __ldg(p.alpha[I] + q);
  cv = load_c<CT>(p.c[I], q, C);  // unrendered texels hold stale values, replaced by 0 below
}

// Stage the footprints of the enabled levels 1..L-1 (entry k of the concatenation
// level 1, level 2, level 3 in round k / MTHR); every load is issued before the first is
// used.  Leaves per warp in sm.any bit I when a staged a_I is positive and bit 4 + I when
// a staged texel of level I is not rendered.
template <typename CT, int C, int L>
__device__ __forceinline__ void stage(const MergeParams& p, MergeSmem<C>& sm, int X0, int Y0) {
  constexpr int N1 = Lv<1>::n, N2 = Lv<2>::n, ROUNDS = (NTAP + MTHR - 1) / MTHR;
  uint8_t st[ROUNDS];
  float av[ROUNDS];
  float3 cv[ROUNDS];
  int lev[ROUNDS];
#pragma unroll
  for (int j = 0; j < ROUNDS; ++j) {
    const int k = threadIdx.x + j * MTHR;
    lev[j] = 0;
    st[j] = 0;
    av[j] = 0.0f;
    cv[j] = make_float3(0.f, 0.f, 0.f);
    if (k < N1) {
      if (L > 1 && p.enabled[1]) {
        load_entry<CT, C, 1>(p, X0, Y0, k, st[j], av[j], cv[j]);
        lev[j] = 1;
      }
    } else if (k < N1 + N2) {
      if (L > 2 && p.enabled[2]) {
        load_entry<CT, C, (L > 2 ? 2 : 1)>(p, X0, Y0, k - N1, st[j], av[j], cv[j]);
        lev[j] = 2;
      }
    } else if (k < NTAP) {
      if (L > 3) {
        load_entry<CT, C, (L > 3 ? 3 : 1)>(p, X0, Y0, k - N1 - N2, st[j], av[j], cv[j]);
        lev[j] = 3;
      }
    }
  }
  int any = 0;
#pragma unroll
  for (int j = 0; j < ROUNDS; ++j) {
    if (lev[j] == 0) continue;
    const int k = threadIdx.x + j * MTHR;
    const bool on = st[j] != 0;
    sm.a[k] = av[j];
    sm.s[k] = on ? 1.0f : 0.0f;
    sm.cz[0][k] = on ? cv[j].x : 0.0f;
    if (C == 4) {
      sm.cz[C == 4 ? 1 : 0][k] = on ? cv[j].y : 0.0f;
      sm.cz[C == 4 ? 2 : 0][k] = on ? cv[j].z : 0.0f;
    }
    if (av[j] > 0.0f) any |= 1 << lev[j];
    if (!on) any |= 16 << lev[j];
  }
  any = __reduce_or_sync(0xffffffffu, any);
  if ((threadIdx.x & 31) == 0) sm.any[threadIdx.x >> 5] = any;
}

// Blend of level I >= 1 into the lane's RPW pixels (FIRST: the coarsest level, taken as
// is).  ALLON: every staged texel of the level is rendered, so the weight sum is exactly 1.
template <int C, int I, bool FIRST>
__device__ __forceinline__ void blend_level(const MergeParams& p, const MergeSmem<C>& sm, int lane, int warp,
                                            bool allon, float (&c)[RPW][3]) {
  constexpr int side = Lv<I>::side, off = lv_off<I>(), o = Lv<I>::o, mask = Lv<I>::mask, NR = Lv<I>::nr;
  const float inv = __int_as_float((127 - I) << 23);  // 2^-I
  const int lx = ((lane - o) >> I) + 1;
  const float fx = (float)((lane - o) & mask) * inv;
  const float gx = 1.0f - fx;
  const int fb = ((RPW * warp - o) >> I) + 1;  // first footprint row of the warp
  const int base = off + fb * side + lx;
  float aL[NR], aR[NR];
  if (!FIRST) {
    uint32_t nz = 0;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      aL[j] = sm.a[base + j * side];
      aR[j] = sm.a[base + j * side + 1];
      nz |= __float_as_uint(aL[j]) | __float_as_uint(aR[j]);
    }
    if (nz == 0u) return;  // every tap +0: alpha = 0 for all the lane's pixels
  }
  const float weight = p.weight[I];
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    // footprint row of the pixel row relative to fb, and its fraction: the same for
    // every warp at levels 1 and 2 (RPW w is a multiple of 2^I); the row offset is 0 at
    // level 3, whose fraction depends on the warp's parity
    const int d = ((rr - o) >> I) - ((-o) >> I);
    const int fyi = I <= 2 ? ((rr - o) & mask) : ((RPW * warp + rr - o) & mask);
    const float fy = (float)fyi * inv;
    const float gy = 1.0f - fy;
    float alpha = 0.0f;
    if (!FIRST) {
      // all four taps +0: ahat = +0 and alpha = 0
      if ((__float_as_uint(aL[d]) | __float_as_uint(aR[d]) | __float_as_uint(aL[d + 1]) |
           __float_as_uint(aR[d + 1])) == 0u)
        continue;
    }
    const float w0 = gx * gy, w1 = fx * gy, w2 = gx * fy, w3 = fx * fy;
    if (!FIRST) {
      float ahat = 0.0f;
      ahat = ahat + w0 * aL[d];
      ahat = ahat + w1 * aR[d];
      ahat = ahat + w2 * aL[d + 1];
      ahat = ahat + w3 * aR[d + 1];
      const float wa = weight * ahat;
      alpha = (1.0f < wa) ? 1.0f : wa;
      if (!(alpha > 0.0f)) continue;
    }
    const int t0 = base + d * side;
    const int idx[4] = {t0, t0 + 1, t0 + side, t0 + side + 1};
    const float w[4] = {w0, w1, w2, w3};
    float n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      n0 = n0 + w[k] * sm.cz[0][idx[k]];
      if (C == 4) {
        n1 = n1 + w[k] * sm.cz[C == 4 ? 1 : 0][idx[k]];
        n2 = n2 + w[k] * sm.cz[C == 4 ? 2 : 0][idx[k]];
      }
    }
    if (!allon) {
      float den = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) den = den + w[k] * sm.s[idx[k]];
      if (den != 1.0f) {
        n0 = n0 / den;
        if (C == 4) {
          n1 = n1 / den;
          n2 = n2 / den;
        }
      }
    }
    if (FIRST) {
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

// The coarsest level when it is level 3 and every staged texel is rendered (the weight sum
// is then exactly 1): a warp's four rows read the same four texels, only the vertical
// weight differs, so the lane reads the taps once and takes two rows at a time in packed
// FP32x2 (each half one correctly rounded multiply or add: the scalar form's bits).
template <int C>
__device__ __forceinline__ void first_level3(const MergeSmem<C>& sm, int lane, int warp, float (&c)[RPW][3]) {
  constexpr int I = 3, side = Lv<3>::side, off = lv_off<3>(), o = Lv<3>::o, mask = Lv<3>::mask;
  constexpr int NCH = C == 4 ? 3 : 1;
  const float inv = 0.125f;  // 2^-3
  const int lx = ((lane - o) >> I) + 1;
  const float fx = (float)((lane - o) & mask) * inv;
  const float gx = 1.0f - fx;
  const int t0 = off + (((RPW * warp - o) >> I) + 1) * side + lx;
  float tap[NCH][4];
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    tap[ch][0] = sm.cz[ch][t0];
    tap[ch][1] = sm.cz[ch][t0 + 1];
    tap[ch][2] = sm.cz[ch][t0 + side];
    tap[ch][3] = sm.cz[ch][t0 + side + 1];
  }
  const float2 gx2 = make_float2(gx, gx), fx2 = make_float2(fx, fx);
#pragma unroll
  for (int rr = 0; rr < RPW; rr += 2) {
    const float2 fy = make_float2((float)((RPW * warp + rr - o) & mask) * inv,
                                  (float)((RPW * warp + rr + 1 - o) & mask) * inv);
    const float2 gy = make_float2(1.0f - fy.x, 1.0f - fy.y);
    const float2 w[4] = {__fmul2_rn(gx2, gy), __fmul2_rn(fx2, gy), __fmul2_rn(gx2, fy), __fmul2_rn(fx2, fy)};
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      float2 n = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 4; ++k) n = __fadd2_rn(n, __fmul2_rn(w[k], make_float2(tap[ch][k], tap[ch][k])));
      c[rr][ch] = n.x;
      c[rr + 1][ch] = n.y;
    }
  }
}

template <typename CT, int C, int L>
__global__ void __launch_bounds__(MTHR) merge_kernel(MergeParams p, float* __restrict__ out) {
  __shared__ MergeSmem<C> sm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int X0 = blockIdx.x * MTX, Y0 = blockIdx.y * MTY;
  const int W = p.W, H = p.H;
  const int x = X0 + lane;
  // level 0 taps first: they need no shared memory
  float a0[RPW];
  uint8_t s0[RPW];
  const bool en0 = p.enabled[0] != 0;
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    const int y = Y0 + RPW * warp + rr;
    a0[rr] = 0.0f;
    s0[rr] = 0;
    if (en0 && x < W && y < H) {
      a0[rr] = __ldg(p.alpha[0] + (size_t)y * W + x);
      s0[rr] = __ldg(p.stencil[0] + (size_t)y * W + x);
    }
  }
  if (L > 1) stage<CT, C, L>(p, sm, X0, Y0);
  __syncthreads();
  if (x >= W) return;
  int any = 0;
#pragma unroll
  for (int k = 0; k < MTHR / 32; ++k) any |= sm.any[k];
  float c[RPW][3] = {};
  // coarsest level first, then the finer enabled levels whose footprint holds a_i > 0
  if (L == 4) {
    if (!(any & 128)) first_level3<C>(sm, lane, warp, c);
    else blend_level<C, (L == 4 ? 3 : 1), true>(p, sm, lane, warp, false, c);
  }
  if (L == 3) blend_level<C, (L == 3 ? 2 : 1), true>(p, sm, lane, warp, !(any & 64), c);
  if (L > 3 && p.enabled[2] && (any & 4)) blend_level<C, (L > 3 ? 2 : 1), false>(p, sm, lane, warp, !(any & 64), c);
  if (L == 2) blend_level<C, 1, true>(p, sm, lane, warp, !(any & 32), c);
  if (L > 2 && p.enabled[1] && (any & 2)) blend_level<C, 1, false>(p, sm, lane, warp, !(any & 32), c);
  if (en0) {
    const bool first = L == 1;
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const int y = Y0 + RPW * warp + rr;
      if (y >= H) break;
      const size_t q = (size_t)y * W + x;
      const float ahat = 0.0f + 1.0f * a0[rr];
      const float wa = p.weight[0] * ahat;
      const float alpha = (1.0f < wa) ? 1.0f : wa;
      if (!first && !(alpha > 0.0f)) continue;
      float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f;
      if (s0[rr]) {
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
  for (int rr = 0; rr < RPW; ++rr) {
    const int y = Y0 + RPW * warp + rr;
    if (y >= H) break;
    const size_t o = (size_t)y * W + x;
    if (C == 4)
      reinterpret_cast<float4*>(out)[o] = make_float4(c[rr][0], c[rr][1], c[rr][2], 0.0f);
    else
      out[o] = c[rr][0];
  }
}

template <typename CT, int C>
__global__ void __launch_bounds__(256) blend0_kernel(Blend0Params p, float* __restrict__ out) {
  const uint32_t n = min(__ldg(p.count), (uint32_t)p.W * (uint32_t)p.H);
  const uint32_t stride = gridDim.x * blockDim.x;
  // two entries per round, every list-aligned read (entry, a_0, c_0) of both issued before
  // the first is used: the read-modify-write of the image is the only dependent access
  for (uint32_t k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < n; k0 += 2 * stride) {
    uint32_t e[2];
    float a[2];
    float3 v[2];
    bool in[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t k = k0 + u * stride;
      in[u] = k < n;
      const uint32_t kk = in[u] ? k : k0;
      e[u] = __ldg(p.list + kk);
      a[u] = __ldg(p.a0c + kk);
      v[u] = load_c<CT>(p.c0c, kk, C);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int x = (int)(e[u] & 0xFFFFu), y = (int)(e[u] >> 16);
      // as the merge kernel blends level 0: one tap of weight 1, a rendered texel
      const float ahat = 0.0f + 1.0f * a[u];
      const float wa = p.weight * ahat;
      const float alpha = (1.0f < wa) ? 1.0f : wa;
      if (!in[u] || x >= p.W || y >= p.H || !(alpha > 0.0f)) continue;
      const float om = 1.0f - alpha;
      const size_t o = (size_t)y * p.W + x;
      if (C == 4) {
        float4* q = reinterpret_cast<float4*>(out) + o;
        const float4 c = *q;
        *q = make_float4(v[u].x * alpha + c.x * om, v[u].y * alpha + c.y * om, v[u].z * alpha + c.z * om, 0.0f);
      } else {
        out[o] = v[u].x * alpha + out[o] * om;
      }
    }
  }
}

// One step of the step-wise blending (Sec. 3.3): level i's composite from the previous
// composite (level j > i).  Texel q of level i sits at u = (2^i q + o_i - o_j) / 2^j in
// level-j texels, whose floor and fraction are exactly n >> j and (n & (2^j - 1)) 2^-j for
// the integer n = 2^i q + o_i - o_j (arithmetic shift: the floor of negative n too); the
// four taps are clamped to level j.  The previous composite is defined at every texel,
// so the interpolation is plain.  Then, where the level blends (BLEND) and S_i(q) = 1,
// alpha = min(w_i a_i(q), 1) and, if alpha > 0, comp = c_i alpha + up (1 - alpha).
// SRC_SUB: the previous composite is the coarsest sub-image itself (storage type CT);
// otherwise float / float4 as written here.
constexpr int CH_TX = 32, CH_TY = 8;  // chain CTA: 32 x 8 threads, CH_R rows per thread

template <typename CT, int C, bool SRC_SUB, int CH_R>
__global__ void __launch_bounds__(CH_TX* CH_TY) chain_kernel(ChainParams p) {
  const int qx = blockIdx.x * CH_TX + threadIdx.x;
  if (qx >= p.Wi) return;
  const int oi = p.i == 0 ? 0 : 1 << (p.i - 1), oj = 1 << (p.j - 1);
  const int mask = (1 << p.j) - 1;
  const float inv = __int_as_float((127 - p.j) << 23);  // 2^-j
  // the column's horizontal taps and weights, shared by its rows
  const int nx = qx * (1 << p.i) + oi - oj;
  const int x0 = nx >> p.j;
  const float fx = (float)(nx & mask) * inv;
  const int xa = min(max(x0, 0), p.Wj - 1), xb = min(max(x0 + 1, 0), p.Wj - 1);
  const float gx = 1.0f - fx;
  const int qy0 = blockIdx.y * CH_TY * CH_R + threadIdx.y;
  // every load of the thread's rows first (rows past the level read its last row)
  float3 t[CH_R][4];
  float av[CH_R];
  uint8_t sv[CH_R];
#pragma unroll
  for (int r = 0; r < CH_R; ++r) {
    const int qy = min(qy0 + r * CH_TY, p.Hi - 1);
    const int ny = qy * (1 << p.i) + oi - oj;
    const int y0 = ny >> p.j;
    const int ya = min(max(y0, 0), p.Hj - 1), yb = min(max(y0 + 1, 0), p.Hj - 1);
    const uint32_t idx[4] = {(uint32_t)(ya * p.Wj + xa), (uint32_t)(ya * p.Wj + xb), (uint32_t)(yb * p.Wj + xa),
                             (uint32_t)(yb * p.Wj + xb)};
#pragma unroll
    for (int k = 0; k < 4; ++k) t[r][k] = SRC_SUB ? load_c<CT>(p.src, idx[k], C) : load_c<float>(p.src, idx[k], C);
    const uint32_t q = (uint32_t)(qy * p.Wi + qx);
    sv[r] = p.blend ? __ldg(p.stencil + q) : (uint8_t)0;
    av[r] = p.blend ? __ldg(p.alpha + q) : 0.0f;
  }
  // level i's own values where it is blended in (issued together)
  float alpha[CH_R];
  float3 v[CH_R];
#pragma unroll
  for (int r = 0; r < CH_R; ++r) {
    const float wa = p.weight * av[r];
    alpha[r] = sv[r] ? ((1.0f < wa) ? 1.0f : wa) : 0.0f;
    v[r] = make_float3(0.0f, 0.0f, 0.0f);
    if (alpha[r] > 0.0f) {
      const int qy = min(qy0 + r * CH_TY, p.Hi - 1);
      v[r] = load_c<CT>(p.c, (uint32_t)(qy * p.Wi + qx), C);
    }
  }
#pragma unroll
  for (int r = 0; r < CH_R; ++r) {
    const int qy = qy0 + r * CH_TY;
    if (qy >= p.Hi) break;
    const int ny = qy * (1 << p.i) + oi - oj;
    const float fy = (float)(ny & mask) * inv;
    const float gy = 1.0f - fy;
    const float w[4] = {gx * gy, fx * gy, gx * fy, fx * fy};
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u0 = u0 + w[k] * t[r][k].x;
      if (C == 4) {
        u1 = u1 + w[k] * t[r][k].y;
        u2 = u2 + w[k] * t[r][k].z;
      }
    }
    if (alpha[r] > 0.0f) {
      const float om = 1.0f - alpha[r];
      u0 = v[r].x * alpha[r] + u0 * om;
      if (C == 4) {
        u1 = v[r].y * alpha[r] + u1 * om;
        u2 = v[r].z * alpha[r] + u2 * om;
      }
    }
    const uint32_t q = (uint32_t)(qy * p.Wi + qx);
    if (C == 4)
      reinterpret_cast<float4*>(p.dst)[q] = make_float4(u0, u1, u2, 0.0f);
    else
      p.dst[q] = u0;
  }
}

template <typename CT, int C, int R>
void launch_chain_r(const ChainParams& p, cudaStream_t s) {
  dim3 grid((p.Wi + CH_TX - 1) / CH_TX, (p.Hi + CH_TY * R - 1) / (CH_TY * R)), block(CH_TX, CH_TY);
  if (p.src_sub)
    chain_kernel<CT, C, true, R><<<grid, block, 0, s>>>(p);
  else
    chain_kernel<CT, C, false, R><<<grid, block, 0, s>>>(p);
}

// Four rows per thread where the level fills the GPU with CTAs to spare; one row per
// thread for the small levels, which would otherwise run a fraction of a wave.
int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <typename CT, int C>
void launch_chain_t(const ChainParams& p, cudaStream_t s) {
  const long blocks4 = (long)((p.Wi + CH_TX - 1) / CH_TX) * ((p.Hi + CH_TY * 4 - 1) / (CH_TY * 4));
  if (blocks4 >= 4L * sm_count())
    launch_chain_r<CT, C, 4>(p, s);
  else
    launch_chain_r<CT, C, 1>(p, s);
}

// Blend of sample-count levels (Sec. 6): every sub-image is [H][W], so only the masks
// are interpolated.  Per pixel, from c' = c_{L-1}(p), over every finer enabled level i
// whose texel (x >> i, y >> i) is rendered: a_i interpolated at p exactly as merge_kernel
// does (taps (p - o_i) >> i, +1, clamped; fraction ((p - o_i) & (2^i - 1)) 2^-i),
// alpha = min(w_i a_i, 1) and, where alpha > 0, c' = c_i(p) alpha + c' (1 - alpha).
template <typename CT, int C>
__global__ void __launch_bounds__(256) merge_samples_kernel(MergeParams p, float* __restrict__ out) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= p.W || y >= p.H) return;
  const size_t pix = (size_t)y * p.W + x;
  const float3 top = load_c<CT>(p.c[p.L - 1], pix, C);
  float c0 = top.x, c1 = top.y, c2 = top.z;
  for (int i = p.L - 2; i >= 0; --i) {
    if (!p.enabled[i]) continue;
    const int Wi = p.Wi[i], Hi = p.Hi[i];
    if (!__ldg(p.stencil[i] + (size_t)(y >> i) * Wi + (x >> i))) continue;
    const int o = i == 0 ? 0 : 1 << (i - 1), mask = (1 << i) - 1;
    const float inv = __int_as_float((127 - i) << 23);  // 2^-i
    const int nx = x - o, ny = y - o;
    const int x0 = nx >> i, y0 = ny >> i;
    const float fx = (float)(nx & mask) * inv, fy = (float)(ny & mask) * inv;
    const int xa = min(max(x0, 0), Wi - 1), xb = min(max(x0 + 1, 0), Wi - 1);
    const int ya = min(max(y0, 0), Hi - 1), yb = min(max(y0 + 1, 0), Hi - 1);
    const float* a = p.alpha[i];
    const float w0 = (1.0f - fx) * (1.0f - fy), w1 = fx * (1.0f - fy), w2 = (1.0f - fx) * fy, w3 = fx * fy;
    float ahat = 0.0f;
    ahat = ahat + w0 * __ldg(a + (size_t)ya * Wi + xa);
    ahat = ahat + w1 * __ldg(a + (size_t)ya * Wi + xb);
    ahat = ahat + w2 * __ldg(a + (size_t)yb * Wi + xa);
    ahat = ahat + w3 * __ldg(a + (size_t)yb * Wi + xb);
    const float wa = p.weight[i] * ahat;
    const float alpha = (1.0f < wa) ? 1.0f : wa;
    if (!(alpha > 0.0f)) continue;
    const float3 v = load_c<CT>(p.c[i], pix, C);
    const float om = 1.0f - alpha;
    c0 = v.x * alpha + c0 * om;
    if (C == 4) {
      c1 = v.y * alpha + c1 * om;
      c2 = v.z * alpha + c2 * om;
    }
  }
  if (C == 4)
    reinterpret_cast<float4*>(out)[pix] = make_float4(c0, c1, c2, 0.0f);
  else
    out[pix] = c0;
}

// Direct upsampling with bilateral taps (merge_mode 2): merge_kernel's arithmetic per
// pixel, except that c_i is interpolated over the rendered taps that lie on the pixel's
// surface, |d(s_i(Q)) - d(p)| <= rel * d(p), falling back to every rendered tap when none
// does.  One pixel per thread; the taps are read from global memory (L1 / L2).
template <typename CT, int C>
__global__ void __launch_bounds__(256) merge_bilateral_kernel(MergeParams p, const float* __restrict__ depth,
                                                               float rel, float* __restrict__ out) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= p.W || y >= p.H) return;
  const size_t pix = (size_t)y * p.W + x;
  const float dp = __ldg(depth + pix);
  const float thr = rel * dp;
  float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
  bool first = true;
  for (int i = p.L - 1; i >= 0; --i) {
    if (!p.enabled[i]) continue;
    const int Wi = p.Wi[i], Hi = p.Hi[i];
    const int o = i == 0 ? 0 : 1 << (i - 1), mask = (1 << i) - 1;
    const float inv = __int_as_float((127 - i) << 23);  // 2^-i
    const int nx = x - o, ny = y - o;
    const int x0 = nx >> i, y0 = ny >> i;
    const float fx = (float)(nx & mask) * inv, fy = (float)(ny & mask) * inv;
    const int xs[2] = {min(max(x0, 0), Wi - 1), min(max(x0 + 1, 0), Wi - 1)};
    const int ys[2] = {min(max(y0, 0), Hi - 1), min(max(y0 + 1, 0), Hi - 1)};
    const float w[4] = {(1.0f - fx) * (1.0f - fy), fx * (1.0f - fy), (1.0f - fx) * fy, fx * fy};
    const int tx[4] = {xs[0], xs[1], xs[0], xs[1]}, ty[4] = {ys[0], ys[0], ys[1], ys[1]};
    float ahat = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) ahat = ahat + w[k] * __ldg(p.alpha[i] + (size_t)ty[k] * Wi + tx[k]);
    const float wa = p.weight[i] * ahat;
    const float alpha = (1.0f < wa) ? 1.0f : wa;
    if (!first && !(alpha > 0.0f)) continue;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, denb = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const size_t q = (size_t)ty[k] * Wi + tx[k];
      if (!__ldg(p.stencil[i] + q)) continue;
      const float3 v = load_c<CT>(p.c[i], q, C);
      n0 = n0 + w[k] * v.x;
      if (C == 4) {
        n1 = n1 + w[k] * v.y;
        n2 = n2 + w[k] * v.z;
      }
      den = den + w[k];
      const int sx = min((tx[k] << i) + o, p.W - 1), sy = min((ty[k] << i) + o, p.H - 1);
      const float dq = __ldg(depth + (size_t)sy * p.W + sx);
      if (!(fabsf(dq - dp) <= thr)) continue;
      b0 = b0 + w[k] * v.x;
      if (C == 4) {
        b1 = b1 + w[k] * v.y;
        b2 = b2 + w[k] * v.z;
      }
      denb = denb + w[k];
    }
    if (denb > 0.0f) {
      n0 = b0;
      n1 = b1;
      n2 = b2;
      den = denb;
    }
    if (first) {
      c0 = n0 / den;
      if (C == 4) {
        c1 = n1 / den;
        c2 = n2 / den;
      }
      first = false;
      continue;
    }
    const float om = 1.0f - alpha;
    c0 = (n0 / den) * alpha + c0 * om;
    if (C == 4) {
      c1 = (n1 / den) * alpha + c1 * om;
      c2 = (n2 / den) * alpha + c2 * om;
    }
  }
  if (C == 4)
    reinterpret_cast<float4*>(out)[pix] = make_float4(c0, c1, c2, 0.0f);
  else
    out[pix] = c0;
}

template <typename CT, int C>
void launch_merge_t(const MergeParams& p, float* out, cudaStream_t s) {
  dim3 grid((p.W + MTX - 1) / MTX, (p.H + MTY - 1) / MTY);
  switch (p.L) {
    case 1: merge_kernel<CT, C, 1><<<grid, MTHR, 0, s>>>(p, out); break;
    case 2: merge_kernel<CT, C, 2><<<grid, MTHR, 0, s>>>(p, out); break;
    case 3: merge_kernel<CT, C, 3><<<grid, MTHR, 0, s>>>(p, out); break;
    default: merge_kernel<CT, C, 4><<<grid, MTHR, 0, s>>>(p, out); break;
  }
}

}  // namespace

int blend0_grid() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = (sms > 0 ? sms : 1) * 8;
  }
  return blocks;
}

cudaError_t launch_blend0(const Blend0Params& p, float* out, cudaStream_t s) {
  const int grid = blend0_grid();
  if (p.C == 4) {
    if (p.half_store) blend0_kernel<__half, 4><<<grid, 256, 0, s>>>(p, out);
    else blend0_kernel<float, 4><<<grid, 256, 0, s>>>(p, out);
  } else {
    if (p.half_store) blend0_kernel<__half, 1><<<grid, 256, 0, s>>>(p, out);
    else blend0_kernel<float, 1><<<grid, 256, 0, s>>>(p, out);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chain(const ChainParams& p, cudaStream_t s) {
  if (p.C == 4) {
    if (p.half_store) launch_chain_t<__half, 4>(p, s);
    else launch_chain_t<float, 4>(p, s);
  } else {
    if (p.half_store) launch_chain_t<__half, 1>(p, s);
    else launch_chain_t<float, 1>(p, s);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_merge_samples(const MergeParams& p, float* out, cudaStream_t s) {
  dim3 grid((p.W + 31) / 32, (p.H + 7) / 8), block(32, 8);
  if (p.C == 4) {
    if (p.half_store) merge_samples_kernel<__half, 4><<<grid, block, 0, s>>>(p, out);
    else merge_samples_kernel<float, 4><<<grid, block, 0, s>>>(p, out);
  } else {
    if (p.half_store) merge_samples_kernel<__half, 1><<<grid, block, 0, s>>>(p, out);
    else merge_samples_kernel<float, 1><<<grid, block, 0, s>>>(p, out);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_merge_bilateral(const MergeParams& p, const float* depth, float rel, float* out, cudaStream_t s) {
  dim3 grid((p.W + 31) / 32, (p.H + 7) / 8), block(32, 8);
  if (p.C == 4) {
    if (p.half_store) merge_bilateral_kernel<__half, 4><<<grid, block, 0, s>>>(p, depth, rel, out);
    else merge_bilateral_kernel<float, 4><<<grid, block, 0, s>>>(p, depth, rel, out);
  } else {
    if (p.half_store) merge_bilateral_kernel<__half, 1><<<grid, block, 0, s>>>(p, depth, rel, out);
    else merge_bilateral_kernel<float, 1><<<grid, block, 0, s>>>(p, depth, rel, out);
  }
  count_launches(1);
  return cudaGetLastError();
}

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
