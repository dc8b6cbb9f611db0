// k_blur.cu -- the bilateral blur of the rendered sub-images (Sec. 4.1).
//
// The paper blurs the SSAO sub-images, above all the coarse ones, to lower the variance
// of the effect, and keeps the blur from taking values out of texels that were never
// rendered.  For every listed texel q of level i:
//   b_i(q) = sum_t w_t c_i(q + t) / sum_t w_t
// over the offsets t of the 5 x 5 window (tx, ty in -2..2, row-major order) whose texel is
// inside the level, in the stencil, and on q's surface:
//   |d(s_i(q + t)) - d(s_i(q))| <= rel * d(s_i(q)),
// d the full-resolution depth at a texel's sample pixel.  w_t = B[tx] B[ty] with the
// binomial row B = (1, 4, 6, 4, 1); each product and sum is one IEEE operation in that
// order (the library builds with -fmad=false), and the quotient is IEEE division.  Every
// texel with its stencil set is blurred; the others are not written.
//
// blur_kernel: one CTA per 32 x 8 tile of level texels, over the tiles of every blurred
// level in one launch.  A tile without a rendered texel returns after reading its
// stencil.  Otherwise the CTA stages the tile's 36 x 12 footprint -- per texel the depth at
// its sample pixel (NaN where the stencil is 0) beside its value -- in shared memory,
// issuing every load before storing any, and each rendered texel then sums its window
// from shared memory in the definition's order, one shared-memory load per tap.
#include "mrr_internal.cuh"

namespace mrr {

namespace {

constexpr int BLUR_THREADS = 256;

// One texel's channels: C = 1 (float / half) or 4 (float4 / half4, the SSGI layout).
template <int C, bool HALF> struct Texel;
template <> struct Texel<1, false> {
  float v[1];
  __device__ __forceinline__ void load(const void* c, size_t i) { v[0] = __ldg(reinterpret_cast<const float*>(c) + i); }
  __device__ __forceinline__ void store(void* c, size_t i) const { reinterpret_cast<float*>(c)[i] = v[0]; }
};
template <> struct Texel<1, true> {
  float v[1];
  __device__ __forceinline__ void load(const void* c, size_t i) {
    v[0] = __half2float(reinterpret_cast<const __half*>(c)[i]);
  }
  __device__ __forceinline__ void store(void* c, size_t i) const {
    reinterpret_cast<__half*>(c)[i] = __float2half_rn(v[0]);
  }
};
template <> struct Texel<4, false> {
  float v[3];
  __device__ __forceinline__ void load(const void* c, size_t i) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(c) + i);
    v[0] = f.x;
    v[1] = f.y;
    v[2] = f.z;
  }
  __device__ __forceinline__ void store(void* c, size_t i) const {
    reinterpret_cast<float4*>(c)[i] = make_float4(v[0], v[1], v[2], 0.0f);
  }
};
template <> struct Texel<4, true> {
  float v[3];
  __device__ __forceinline__ void load(const void* c, size_t i) {
    const half4 h = reinterpret_cast<const half4*>(c)[i];
    v[0] = __half2float(h.x);
    v[1] = __half2float(h.y);
    v[2] = __half2float(h.z);
  }
  __device__ __forceinline__ void store(void* c, size_t i) const {
    half4 h;
    h.x = __float2half_rn(v[0]);
    h.y = __float2half_rn(v[1]);
    h.z = __float2half_rn(v[2]);
    h.w = __float2half_rn(0.0f);
    reinterpret_cast<half4*>(c)[i] = h;
  }
};

__device__ __forceinline__ float binomial(int t) { return t == 0 ? 6.0f : (t == 1 || t == -1) ? 4.0f : 1.0f; }

constexpr int BTX = 32, BTY = 8, BH = 2;                 // tile of level texels, window halo
constexpr int BSX = BTX + 2 * BH, BSY = BTY + 2 * BH;    // staged footprint
constexpr int BN = BSX * BSY;
constexpr int BROUNDS = (BN + BLUR_THREADS - 1) / BLUR_THREADS;
static_assert(BTX * BTY == BLUR_THREADS, "one thread per tile texel");

// Staged footprint entry: the depth at the texel's sample pixel, then the value.  A texel
// outside the stencil or the level holds a NaN depth instead: |NaN - d| <= thr is false,
// so it drops out of the sums exactly as the definition's skipped term (a NaN input depth
// behaves the same on both sides).
template <int NC> struct BlurEntry;
template <> struct BlurEntry<1> { using T = float2; };
template <> struct BlurEntry<3> { using T = float4; };

template <int C, bool HALF>
__global__ void __launch_bounds__(BLUR_THREADS) blur_kernel(BlurParams p) {
  constexpr int NC = C == 1 ? 1 : 3;
  using E = typename BlurEntry<NC>::T;
  __shared__ E sm[BN];
  int k = 0;
#pragma unroll
  for (int j = 1; j < MRR_MAX_LEVELS; ++j)
    if (j < p.nlev && (int)blockIdx.x >= p.tile_begin[j]) k = j;
  const int i = p.level[k], Wi = p.Wi[k], Hi = p.Hi[k];
  const int t = (int)blockIdx.x - p.tile_begin[k];
  const int gx = (Wi + BTX - 1) / BTX;
  const int X0 = (t % gx) * BTX, Y0 = (t / gx) * BTY;
  const int tx = threadIdx.x % BTX, ty = threadIdx.x / BTX;
  const int qx = X0 + tx, qy = Y0 + ty;
  const uint8_t* S = p.stencil[k];
  const bool mine = qx < Wi && qy < Hi && __ldg(S + (size_t)qy * Wi + qx) != 0;
  if (!__syncthreads_or(mine)) return;  // no rendered texel in the tile
  // stage the footprint: every load of both rounds is issued before the first is stored;
  // entries outside the level read the nearest texel and are marked unrendered
  const int o = i == 0 ? 0 : 1 << (i - 1);
  uint8_t st[BROUNDS];
  float dv[BROUNDS];
  Texel<C, HALF> cv[BROUNDS];
#pragma unroll
  for (int r = 0; r < BROUNDS; ++r) {
    const int e = threadIdx.x + r * BLUR_THREADS;
    st[r] = 0;
    dv[r] = 0.0f;
#pragma unroll
    for (int ch = 0; ch < NC; ++ch) cv[r].v[ch] = 0.0f;
    if (e < BN) {
      const int ly = e / BSX, lx = e - ly * BSX;
      const int ux = X0 - BH + lx, uy = Y0 - BH + ly;
      const int cx = min(max(ux, 0), Wi - 1), cy = min(max(uy, 0), Hi - 1);
      const size_t u = (size_t)cy * Wi + cx;
      const uint8_t sv = __ldg(S + u);
      st[r] = (ux == cx && uy == cy) ? sv : (uint8_t)0;
      // sample pixel s_i = min(2^i q + o_i, n - 1)
      const int sx = min(cx * (1 << i) + o, p.W - 1), sy = min(cy * (1 << i) + o, p.H - 1);
      dv[r] = __ldg(p.depth + (size_t)sy * p.W + sx);
      cv[r].load(p.c[k], u);
    }
  }
#pragma unroll
  for (int r = 0; r < BROUNDS; ++r) {
    const int e = threadIdx.x + r * BLUR_THREADS;
    if (e < BN) {
      const float d = st[r] ? dv[r] : __int_as_float(0x7fc00000);
      E v;
      if constexpr (NC == 1) {
        v = make_float2(d, cv[r].v[0]);
      } else {
        v = make_float4(d, cv[r].v[0], cv[r].v[1], cv[r].v[2]);
      }
      sm[e] = v;
    }
  }
  __syncthreads();
  if (!mine) return;
  const int ctr = (ty + BH) * BSX + tx + BH;
  const float d = sm[ctr].x;
  const float thr = p.rel * d;
  float num[NC], den = 0.0f;
#pragma unroll
  for (int ch = 0; ch < NC; ++ch) num[ch] = 0.0f;
#pragma unroll
  for (int wy = 0; wy < 5; ++wy) {
    const float by = binomial(wy - 2);
#pragma unroll
    for (int wx = 0; wx < 5; ++wx) {
      const E v = sm[ctr + (wy - 2) * BSX + (wx - 2)];
      // taps in the window's row-major order; a tap that fails adds nothing, exactly as
      // the definition's skipped term
      if (fabsf(v.x - d) <= thr) {
        const float w = by * binomial(wx - 2);
        if constexpr (NC == 1) {
          num[0] = num[0] + w * v.y;
        } else {
          num[0] = num[0] + w * v.y;
          num[1] = num[1] + w * v.z;
          num[2] = num[2] + w * v.w;
        }
        den = den + w;
      }
    }
  }
  Texel<C, HALF> out;
#pragma unroll
  for (int ch = 0; ch < NC; ++ch) out.v[ch] = num[ch] / den;
  out.store(p.b[k], (size_t)qy * Wi + qx);
}

}  // namespace

int blur_tiles(int Wi, int Hi) { return ((Wi + BTX - 1) / BTX) * ((Hi + BTY - 1) / BTY); }

cudaError_t launch_blur(const BlurParams& p, cudaStream_t s) {
  if (p.nlev == 0) return cudaSuccess;
  const int grid = p.tile_begin[p.nlev];
  if (p.C == 1) {
    if (p.half_store)
      blur_kernel<1, true><<<grid, BLUR_THREADS, 0, s>>>(p);
    else
      blur_kernel<1, false><<<grid, BLUR_THREADS, 0, s>>>(p);
  } else {
    if (p.half_store)
      blur_kernel<4, true><<<grid, BLUR_THREADS, 0, s>>>(p);
    else
      blur_kernel<4, false><<<grid, BLUR_THREADS, 0, s>>>(p);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
