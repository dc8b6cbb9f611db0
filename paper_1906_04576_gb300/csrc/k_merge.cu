// k_merge.cu -- upsampling and blending of the sub-images (Sec. 4.2, Eq. (1)).
//
// merge_kernel: a thread owns a block of 4 x BH full-resolution pixels at (4a, BH b) (BH = 4,
// or 2 for three-channel images).  Level texel q sits at full-resolution position
// 2^i q + o_i, so pixel p reads level coordinate u = (p - o_i) / 2^i: taps floor(u) and
// floor(u) + 1, clamped to the level, with the fraction ((p - o_i) & (2^i - 1)) 2^-i.  Over
// a block the taps of every level lie in a window of at most 3 x 3 texels, and which window
// slot a pixel starts at depends only on its place in the block (the block's phase modulo
// 2^i changes the fractions, never the slots).  The thread reads each level's window once
// into registers -- a_i, the stencil as 0/1 and c_i with unrendered texels replaced by 0 --
// and interpolates separably: first along x for every window row, then along y, for â_i
// (plain), and for the numerator and denominator of the masked bilinear ĉ_i (rendered taps
// only, weights renormalised).  Per pixel, from the coarsest level down: alpha =
// min(w_i â_i, 1) where â_i > 0 and c' = c' + alpha (ĉ_i - c'); the coarsest level is taken
// as is.  A level none of whose window texels has a_i > 0 leaves the block unchanged.
// Level 0, when the merge blends it (the staged path), is one tap of weight 1 per pixel,
// blended exactly as blend0_kernel blends it from level 0's list on the frame path.
// The interpolation differs from the oracle's four-weight sum only in rounding; the
// discrete step (whether â_i > 0) is the same, since every tap and weight is non-negative.
//
// chain_kernel: the step-wise reading of Sec. 3.3 instead -- one launch per step, each
// level's composite computed at its own resolution from the previous one.
// merge_samples_kernel: the blend of sample-count levels (full-resolution sub-images).
// merge_bilateral_kernel: the direct merge with depth-aware (bilateral) taps.
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

// ---- merge_kernel
constexpr int MG_TX = 32, MG_TY = 4;  // threads per CTA: 32 blocks across, 4 down
template <int C> constexpr int mg_bh() { return C == 4 ? 2 : 4; }  // block height (pixels)

// One axis of a level-I window for a block of B pixels starting at a multiple of 4 (x) or
// of B (y): slot(c) = the window slot of pixel c's first tap, nt() = window size.  The slots
// are the same for every phase of the block start modulo 2^I (checked by nt_ok below).
template <int I, int B> struct MgAxis {
  static constexpr int o = I == 0 ? 0 : (1 << (I - 1));
  static constexpr int S = 1 << I;
  static constexpr int fl(int v) { return v >= 0 ? v / S : -((-v + S - 1) / S); }  // floor(v / 2^I)
  // phase ph = block start modulo 2^I
  static constexpr int slot_ph(int ph, int c) { return fl(ph + c - o) - fl(ph - o); }
  static constexpr int frac_ph(int ph, int c) { return (ph + c - o) - fl(ph + c - o) * S; }
  static constexpr int slot(int c) { return slot_ph(0, c); }
  static constexpr int nt() {
    int m = 0;
    for (int ph = 0; ph < S; ph += (B < S ? B : S))
      for (int c = 0; c < B; ++c) {
        const int e = slot_ph(ph, c) + (frac_ph(ph, c) > 0 ? 1 : 0);
        m = e > m ? e : m;
      }
    return m + 1;
  }
  static constexpr bool slots_fixed() {
    for (int ph = 0; ph < S; ph += (B < S ? B : S))
      for (int c = 0; c < B; ++c)
        if (slot_ph(ph, c) != slot_ph(0, c)) return false;
    return true;
  }
  // every block start is a multiple of B (and of 4 along x), so the phase is 0 when 2^I <= B
  static constexpr bool frac_fixed() { return S <= B; }
};
static_assert(MgAxis<1, 4>::nt() == 3 && MgAxis<2, 4>::nt() == 3 && MgAxis<3, 4>::nt() == 2, "windows");
static_assert(MgAxis<1, 2>::nt() == 2 && MgAxis<2, 2>::nt() == 2 && MgAxis<3, 2>::nt() == 2, "windows");
static_assert(MgAxis<3, 4>::slots_fixed() && MgAxis<3, 2>::slots_fixed() && MgAxis<2, 2>::slots_fixed(), "slots");

// The fraction of pixel c of a block starting at X0 (a multiple of B) at level I.
template <int I, int B>
__device__ __forceinline__ float mg_frac(int X0, int c) {
  using A = MgAxis<I, B>;
  if (A::frac_fixed()) return (float)A::frac_ph(0, c) * (1.0f / (float)A::S);
  return (float)((X0 + c - A::o) & (A::S - 1)) * (1.0f / (float)A::S);
}

__device__ __forceinline__ float mg_lerp(float a, float b, float f) { return fmaf(f, b - a, a); }

// Interpolation of one level's window over the block and the blend of Eq. (1).  MASKED:
// some window tap is not rendered, so the denominator of the masked bilinear varies.
template <int I, int BH, int NX, int NY, int NCH, bool FIRST, bool MASKED>
__device__ __forceinline__ void mg_blend(const MergeParams& p, int X0, int Y0, const float (&tA)[NY][NX],
                                         const float (&tD)[NY][NX], const float (&tN)[NY][NX][NCH],
                                         float (&cc)[BH][4][NCH]) {
  using AX = MgAxis<I, 4>;
  using AY = MgAxis<I, BH>;
  // along x, every window row
  float hA[NY][4], hD[NY][4], hN[NY][4][NCH];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = AX::slot(c);
    const int j1 = j + 1 < NX ? j + 1 : NX - 1;
    const float f = mg_frac<I, 4>(X0, c);
    const bool fixed0 = AX::frac_fixed() && AX::frac_ph(0, c) == 0;
#pragma unroll
    for (int r = 0; r < NY; ++r) {
      if (fixed0) {
        if (!FIRST) hA[r][c] = tA[r][j];
        if (MASKED) hD[r][c] = tD[r][j];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) hN[r][c][ch] = tN[r][j][ch];
      } else {
        if (!FIRST) hA[r][c] = mg_lerp(tA[r][j], tA[r][j1], f);
        if (MASKED) hD[r][c] = mg_lerp(tD[r][j], tD[r][j1], f);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) hN[r][c][ch] = mg_lerp(tN[r][j][ch], tN[r][j1][ch], f);
      }
    }
  }
  // along y, and the blend
  const float weight = p.weight[I];
#pragma unroll
  for (int rr = 0; rr < BH; ++rr) {
    const int j = AY::slot(rr);
    const int j1 = j + 1 < NY ? j + 1 : NY - 1;
    const float f = mg_frac<I, BH>(Y0, rr);
    const bool fixed0 = AY::frac_fixed() && AY::frac_ph(0, rr) == 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float ah = 0.0f, den = 1.0f, num[NCH];
      if (fixed0) {
        if (!FIRST) ah = hA[j][c];
        if (MASKED) den = hD[j][c];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) num[ch] = hN[j][c][ch];
      } else {
        if (!FIRST) ah = mg_lerp(hA[j][c], hA[j1][c], f);
        if (MASKED) den = mg_lerp(hD[j][c], hD[j1][c], f);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) num[ch] = mg_lerp(hN[j][c][ch], hN[j1][c][ch], f);
      }
      if (MASKED) {
        // no rendered tap of positive weight: a_hat is 0 there too (a > 0 only where S = 1)
        const float inv = den > 0.0f ? __fdividef(1.0f, den) : 0.0f;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) num[ch] = den == 1.0f ? num[ch] : num[ch] * inv;
      }
      if (FIRST) {
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) cc[rr][c][ch] = num[ch];
      } else {
        const float alpha = __saturatef(weight * ah);  // min(w a_hat, 1), a_hat >= 0
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) cc[rr][c][ch] = fmaf(alpha, num[ch] - cc[rr][c][ch], cc[rr][c][ch]);
      }
    }
  }
}

// Level I >= 1 over the thread's block (FIRST: the coarsest level, which sets c').
template <typename CT, int C, int I, int BH, bool FIRST>
__device__ __forceinline__ void mg_level(const MergeParams& p, int X0, int Y0, float (&cc)[BH][4][C == 4 ? 3 : 1]) {
  constexpr int NCH = C == 4 ? 3 : 1;
  using AX = MgAxis<I, 4>;
  using AY = MgAxis<I, BH>;
  constexpr int NX = AX::nt(), NY = AY::nt();
  const int Wi = p.Wi[I], Hi = p.Hi[I];
  const int bx = (X0 - AX::o) >> I, by = (Y0 - AY::o) >> I;  // arithmetic shifts: floors
  int xs[NX], ys[NY];
#pragma unroll
  for (int j = 0; j < NX; ++j) xs[j] = min(max(bx + j, 0), Wi - 1);
#pragma unroll
  for (int j = 0; j < NY; ++j) ys[j] = min(max(by + j, 0), Hi - 1);
  float tA[NY][NX], tD[NY][NX], tN[NY][NX][NCH];
  uint8_t st[NY][NX];
  float3 cv[NY][NX];
#pragma unroll
  for (int r = 0; r < NY; ++r)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const size_t q = (size_t)ys[r] * Wi + xs[j];
      st[r][j] = __ldg(p.stencil[I] + q);
      tA[r][j] = FIRST ? 0.0f : __ldg(p.alpha[I] + q);
      cv[r][j] = load_c<CT>(p.c[I], q, C);  // stale where not rendered: replaced by 0 below
    }
  if (!FIRST) {
    uint32_t nz = 0u;
#pragma unroll
    for (int r = 0; r < NY; ++r)
#pragma unroll
      for (int j = 0; j < NX; ++j) nz |= __float_as_uint(tA[r][j]);
    if (nz == 0u) return;  // a_i = 0 over the window: alpha = 0 for the whole block
  }
  bool allon = true;
#pragma unroll
  for (int r = 0; r < NY; ++r)
#pragma unroll
    for (int j = 0; j < NX; ++j) allon = allon && st[r][j] != 0;
  if (allon) {
    // every tap rendered: the weight sum is exactly 1, so c_hat is the plain interpolation,
    // and alpha = sat(w a_hat) blends every pixel (alpha = 0 leaves c' unchanged exactly)
#pragma unroll
    for (int r = 0; r < NY; ++r)
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        tN[r][j][0] = cv[r][j].x;
        if (NCH == 3) {
          tN[r][j][NCH == 3 ? 1 : 0] = cv[r][j].y;
          tN[r][j][NCH == 3 ? 2 : 0] = cv[r][j].z;
        }
      }
    mg_blend<I, BH, NX, NY, NCH, FIRST, false>(p, X0, Y0, tA, tD, tN, cc);
  } else {
#pragma unroll
    for (int r = 0; r < NY; ++r)
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        const bool on = st[r][j] != 0;
        tD[r][j] = on ? 1.0f : 0.0f;
        tN[r][j][0] = on ? cv[r][j].x : 0.0f;
        if (NCH == 3) {
          tN[r][j][NCH == 3 ? 1 : 0] = on ? cv[r][j].y : 0.0f;
          tN[r][j][NCH == 3 ? 2 : 0] = on ? cv[r][j].z : 0.0f;
        }
      }
    mg_blend<I, BH, NX, NY, NCH, FIRST, true>(p, X0, Y0, tA, tD, tN, cc);
  }
}

template <typename CT, int C, int L>
__global__ void __launch_bounds__(MG_TX* MG_TY) merge_kernel(MergeParams p, float* __restrict__ out, int vec) {
  constexpr int BH = mg_bh<C>(), NCH = C == 4 ? 3 : 1;
  const int X0 = 4 * (int)(blockIdx.x * MG_TX + threadIdx.x);
  const int Y0 = BH * (int)(blockIdx.y * MG_TY + threadIdx.y);
  const int W = p.W, H = p.H;
  if (X0 >= W || Y0 >= H) return;
  float cc[BH][4][NCH];
  // coarsest level first (always blended), then every finer enabled level above 0
  if (L == 4) mg_level<CT, C, (L == 4 ? 3 : 1), BH, true>(p, X0, Y0, cc);
  if (L == 3) mg_level<CT, C, (L == 3 ? 2 : 1), BH, true>(p, X0, Y0, cc);
  if (L == 2) mg_level<CT, C, 1, BH, true>(p, X0, Y0, cc);
  if (L > 3 && p.enabled[2]) mg_level<CT, C, 2, BH, false>(p, X0, Y0, cc);
  if (L > 2 && p.enabled[1]) mg_level<CT, C, 1, BH, false>(p, X0, Y0, cc);
  if (L == 1 || p.enabled[0]) {
    // level 0: one tap of weight 1 per pixel, blended as blend0_kernel does
#pragma unroll
    for (int rr = 0; rr < BH; ++rr) {
      const int y = Y0 + rr;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int x = X0 + c;
        if (y >= H || x >= W) continue;
        const size_t q = (size_t)y * W + x;
        const float a0 = __ldg(p.alpha[0] + q);
        const bool s0 = __ldg(p.stencil[0] + q) != 0;
        const float3 v = s0 ? load_c<CT>(p.c[0], q, C) : make_float3(0.f, 0.f, 0.f);
        const float vv[3] = {v.x, v.y, v.z};
        if (L == 1) {
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) cc[rr][c][ch] = s0 ? vv[ch] : __int_as_float(0x7fc00000);
          continue;
        }
        const float ahat = 0.0f + 1.0f * a0;
        const float wa = p.weight[0] * ahat;
        const float alpha = (1.0f < wa) ? 1.0f : wa;
        if (!(alpha > 0.0f)) continue;
        const float om = 1.0f - alpha;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          // no rendered tap: 0/0, as the definition gives (cannot happen where alpha > 0)
          const float n = s0 ? vv[ch] : __int_as_float(0x7fc00000);
          cc[rr][c][ch] = n * alpha + cc[rr][c][ch] * om;
        }
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < BH; ++rr) {
    const int y = Y0 + rr;
    if (y >= H) break;
    const size_t o = (size_t)y * W + X0;
    if (C == 4) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (X0 + c < W)
          reinterpret_cast<float4*>(out)[o + c] =
              make_float4(cc[rr][c][0], cc[rr][c][NCH == 3 ? 1 : 0], cc[rr][c][NCH == 3 ? 2 : 0], 0.0f);
    } else if (vec && X0 + 3 < W) {
      *reinterpret_cast<float4*>(out + o) = make_float4(cc[rr][0][0], cc[rr][1][0], cc[rr][2][0], cc[rr][3][0]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (X0 + c < W) out[o + c] = cc[rr][c][0];
    }
  }
}

// The recomposition of the disjoint-tile ablation: pixel p takes the sub-image of the
// finest enabled level whose stencil covers it, interpolated bilinearly at p over that
// level's rendered taps of positive weight (weights renormalised), with no blending; NaN
// where no level covers p or the covering level has no such tap.  Weights and sums as the
// direct merge's definition: products of the axis weights, taps in order, IEEE division.
template <typename CT, int C>
__global__ void __launch_bounds__(256) merge_disjoint_kernel(MergeParams p, float* __restrict__ out) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= p.W || y >= p.H) return;
  const float nan = __int_as_float(0x7fc00000);
  float v[3] = {nan, nan, nan};
  for (int i = 0; i < p.L; ++i) {
    if (!p.enabled[i]) continue;
    const int Wi = p.Wi[i], Hi = p.Hi[i];
    if (!__ldg(p.stencil[i] + (size_t)(y >> i) * Wi + (x >> i))) continue;
    const int o = i == 0 ? 0 : (1 << (i - 1)), mask = (1 << i) - 1;
    const float inv = __int_as_float((127 - i) << 23);  // 2^-i
    const int nx = x - o, ny = y - o;
    const int x0 = nx >> i, y0 = ny >> i;  // arithmetic shifts: floors
    const float fx = (float)(nx & mask) * inv, fy = (float)(ny & mask) * inv;
    const int xs[2] = {min(max(x0, 0), Wi - 1), min(max(x0 + 1, 0), Wi - 1)};
    const int ys[2] = {min(max(y0, 0), Hi - 1), min(max(y0 + 1, 0), Hi - 1)};
    const float w[4] = {(1.0f - fx) * (1.0f - fy), fx * (1.0f - fy), (1.0f - fx) * fy, fx * fy};
    float num[3] = {0.f, 0.f, 0.f}, den = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const size_t q = (size_t)ys[k >> 1] * Wi + xs[k & 1];
      if (!__ldg(p.stencil[i] + q) || !(w[k] > 0.0f)) continue;
      const float3 cv = load_c<CT>(p.c[i], q, C);
      num[0] = num[0] + w[k] * cv.x;
      num[1] = num[1] + w[k] * cv.y;
      num[2] = num[2] + w[k] * cv.z;
      den = den + w[k];
    }
    if (den > 0.0f) {
      v[0] = num[0] / den;
      v[1] = num[1] / den;
      v[2] = num[2] / den;
    }
    break;
  }
  const size_t pix = (size_t)y * p.W + x;
  if (C == 4)
    reinterpret_cast<float4*>(out)[pix] = make_float4(v[0], v[1], v[2], 0.0f);
  else
    out[pix] = v[0];
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
      // alpha = 1: v 1 + c 0 is v itself (c' is finite and the effects' values are
      // non-negative, never -0), so the image is written without being read
      if (C == 4) {
        float4* q = reinterpret_cast<float4*>(out) + o;
        if (alpha == 1.0f) {
          *q = make_float4(v[u].x, v[u].y, v[u].z, 0.0f);
        } else {
          const float4 c = *q;
          *q = make_float4(v[u].x * alpha + c.x * om, v[u].y * alpha + c.y * om, v[u].z * alpha + c.z * om, 0.0f);
        }
      } else {
        out[o] = alpha == 1.0f ? v[u].x : v[u].x * alpha + out[o] * om;
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
  constexpr int BH = mg_bh<C>();
  const int bw = (p.W + 3) / 4, bh = (p.H + BH - 1) / BH;
  dim3 grid((bw + MG_TX - 1) / MG_TX, (bh + MG_TY - 1) / MG_TY), block(MG_TX, MG_TY);
  // four pixels per 16-byte store when every row starts on a 16-byte boundary
  const int vec = (p.W % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  switch (p.L) {
    case 1: merge_kernel<CT, C, 1><<<grid, block, 0, s>>>(p, out, vec); break;
    case 2: merge_kernel<CT, C, 2><<<grid, block, 0, s>>>(p, out, vec); break;
    case 3: merge_kernel<CT, C, 3><<<grid, block, 0, s>>>(p, out, vec); break;
    default: merge_kernel<CT, C, 4><<<grid, block, 0, s>>>(p, out, vec); break;
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

cudaError_t launch_merge_disjoint(const MergeParams& p, float* out, cudaStream_t s) {
  dim3 grid((p.W + 31) / 32, (p.H + 7) / 8), block(32, 8);
  if (p.C == 4) {
    if (p.half_store) merge_disjoint_kernel<__half, 4><<<grid, block, 0, s>>>(p, out);
    else merge_disjoint_kernel<float, 4><<<grid, block, 0, s>>>(p, out);
  } else {
    if (p.half_store) merge_disjoint_kernel<__half, 1><<<grid, block, 0, s>>>(p, out);
    else merge_disjoint_kernel<float, 1><<<grid, block, 0, s>>>(p, out);
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
