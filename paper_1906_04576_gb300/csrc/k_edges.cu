// k_edges.cu -- the edge image of Sec. 3.1.
//
// edges_direct_kernel and edges_kernel: one CTA per 32x8 pixel tile.
// edges_direct_kernel (SSAO, SSGI): each lane reads its pixel and its 4 neighbours
//   straight from global memory; the neighbours' lines are the block's own rows, so
//   they are L1 hits and DRAM sees each G-buffer texel about once.
// edges_tma_kernel (rows a multiple of 16 bytes): a persistent CTA walks
//   32x16 output tiles; the tile's depth and normals plus a one-pixel halo arrive by TMA
//   into a ring of two shared-memory stages, the next tile's loads in flight while one
//   is tested (several such CTAs per SM).  Same tests and arithmetic as
//   edges_direct_kernel, read from shared memory.
// Soft shadows, rows a multiple of 16 bytes: shadow_bits_kernel writes the one-sample
//   hard shadow of Sec. 3.1 of every pixel as bits (a reconstruction, a light-space
//   projection and a shadow-map read per pixel), then edges_tma_kernel<NT, true> adds the
//   comparisons of those bits with the in-image neighbours' to its tests.
// edges_kernel (soft shadows, other rows): the tile and a one-pixel halo of depth, normals
//   and the hard shadows are staged in shared memory, so each staged texel's hard shadow
//   is computed once, not once per neighbour test.
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "mrr_internal.cuh"
#include "shade_common.cuh"
#include "tma.cuh"

namespace mrr {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int SX = TX + 2, SY = TY + 2;

// Words a frame's later kernels need at zero (the mask kernel's look-back state), set by
// whichever edge kernel runs first in the frame; the grid-stride covers any grid shape.
__device__ __forceinline__ void zero_words(const EdgeParams& p) {
  if (!p.zero) return;
  const int nthr = gridDim.x * gridDim.y * blockDim.x * blockDim.y;
  const int tid = ((blockIdx.y * gridDim.x + blockIdx.x) * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  for (int i = tid; i < p.zero_words; i += nthr) p.zero[i] = 0u;
}

// Store the edge flag e of pixel (x, y): one byte per pixel, or -- bit-packed output --
// one ballot per 32 pixels of a row (bit b of word w = pixel 32 w + b; bits past the
// image's last column are 0).  All 32 lanes of the warp call it together for one row y
// with x = x0 + lane, x0 a multiple of 32; `valid` is false outside the image.
__device__ __forceinline__ void store_edge(const EdgeParams& p, uint8_t* E, int x, int y, bool valid, bool e) {
  if (p.ebits) {
    const uint32_t b = __ballot_sync(0xffffffffu, valid && e);
    if ((threadIdx.x & 31) == 0 && x < p.v.W && y < p.v.H) p.ebits[(size_t)y * p.ewords + (x >> 5)] = b;
  } else if (valid) {
    E[(size_t)y * p.v.W + x] = e ? 1 : 0;
  }
}

template <typename NT, typename SMT>
__global__ void __launch_bounds__(TX* TY) edges_kernel(EdgeParams p, const float* __restrict__ depth,
                                                        const NT* __restrict__ normal,
                                                        const SMT* __restrict__ smap, uint8_t* __restrict__ E) {
  __shared__ float sd[SY][SX];
  __shared__ float snx[SY][SX], sny[SY][SX], snz[SY][SX];
  __shared__ uint8_t shs[SY][SX];
  zero_words(p);
  const int W = p.v.W, H = p.v.H;
  const int x0 = blockIdx.x * TX - 1, y0 = blockIdx.y * TY - 1;
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int k = tid; k < SX * SY; k += TX * TY) {
    const int ly = k / SX, lx = k - ly * SX;
    const int x = x0 + lx, y = y0 + ly;
    float d = -1.0f;  // outside the image
    float3 n = make_float3(0.f, 0.f, 0.f);
    uint8_t hs = 1;
    if (x >= 0 && x < W && y >= 0 && y < H) {
      const size_t i = (size_t)y * W + x;
      d = __ldg(depth + i);
      n = load_normal(normal, i);
      if (p.ssm && d < p.v.farp) hs = (uint8_t)hard_shadow(p.v, p.L, p.shadow_bias, smap, x, y, d);
    }
    sd[ly][lx] = d;
    snx[ly][lx] = n.x;
    sny[ly][lx] = n.y;
    snz[ly][lx] = n.z;
    shs[ly][lx] = hs;
  }
  __syncthreads();
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  const bool valid = x < W && y < H;
  const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
  const float d = sd[ly][lx];
  // Every staged entry the tests read exists (the footprint covers the 4-neighbourhood),
  // so all of them are evaluated and combined with non-short-circuit & and |: the same
  // decision as testing them in turn, without branches.
  const int ox[4] = {-1, 1, 0, 0}, oy[4] = {0, 0, -1, 1};
  const float nx = snx[ly][lx], ny = sny[ly][lx], nz = snz[ly][lx];
  const uint8_t hs = shs[ly][lx];
  const bool ssm = p.ssm != 0;
  bool e = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float dn = sd[ly + oy[k]][lx + ox[k]];
    const bool in = !(dn < 0.0f);  // a neighbour inside the image
    const bool sky = dn >= p.v.farp;
    const float dot = nx * snx[ly + oy[k]][lx + ox[k]] + ny * sny[ly + oy[k]][lx + ox[k]] +
                      nz * snz[ly + oy[k]][lx + ox[k]];
    e = e | (in & (sky | (dot < p.normal_cos) | (ssm & (shs[ly + oy[k]][lx + ox[k]] != hs))));
  }
  const float thr = p.depth_rel * d;
  const float lapx = (sd[ly][lx - 1] + sd[ly][lx + 1]) - 2.0f * d;
  const float lapy = (sd[ly - 1][lx] + sd[ly + 1][lx]) - 2.0f * d;
  e = e | ((x > 0) & (x < W - 1) & (fabsf(lapx) > thr)) | ((y > 0) & (y < H - 1) & (fabsf(lapy) > thr));
  e = e & valid & (d < p.v.farp);
  store_edge(p, E, x, y, valid, e);
}

// edges_direct_kernel: a lane owns a column of ER vertically adjacent pixels.  Every
// load it needs -- the column rows y0-1 .. y0+ER and the left/right neighbours of its
// pixels, at clamped addresses -- is issued before any of them is used, so a warp waits
// for memory once, and the column values double as up/down neighbours.
constexpr int ER = 2;

template <typename NT>
__global__ void __launch_bounds__(TX* TY) edges_direct_kernel(EdgeParams p, const float* __restrict__ depth,
                                                               const NT* __restrict__ normal,
                                                               uint8_t* __restrict__ E) {
  zero_words(p);
  const int W = p.v.W, H = p.v.H;
  const int x = blockIdx.x * TX + threadIdx.x;
  const int y0 = (blockIdx.y * TY + threadIdx.y) * ER;
  // lanes past the right edge read the last column and store nothing (every lane of the
  // warp reaches the bit-packed store)
  const int xc = min(x, W - 1);
  const float farp = p.v.farp;
  const int xl = max(xc - 1, 0), xr = min(xc + 1, W - 1);
  float dc[ER + 2], dl[ER], dr[ER];
  float3 nc[ER + 2], nl[ER], nr[ER];
#pragma unroll
  for (int r = -1; r <= ER; ++r) {
    const int y = min(max(y0 + r, 0), H - 1);
    dc[r + 1] = __ldg(depth + y * W + xc);
    nc[r + 1] = load_normal(normal, y * W + xc);
  }
#pragma unroll
  for (int r = 0; r < ER; ++r) {
    const int y = min(y0 + r, H - 1);
    dl[r] = __ldg(depth + y * W + xl);
    dr[r] = __ldg(depth + y * W + xr);
    nl[r] = load_normal(normal, y * W + xl);
    nr[r] = load_normal(normal, y * W + xr);
  }
#pragma unroll
  for (int r = 0; r < ER; ++r) {
    const int y = y0 + r;
    const bool valid = x < W && y < H;
    const float d = dc[r + 1];
    uint8_t e = 0;
    if (valid && d < farp) {
      const float3 n = nc[r + 1];
      const bool has[4] = {x > 0, x < W - 1, y > 0, y < H - 1};
      const float dn[4] = {dl[r], dr[r], dc[r], dc[r + 2]};
      const float3 nn[4] = {nl[r], nr[r], nc[r], nc[r + 2]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!has[k]) continue;
        if (dn[k] >= farp) {  // sky neighbour
          e = 1;
          continue;
        }
        if (n.x * nn[k].x + n.y * nn[k].y + n.z * nn[k].z < p.normal_cos) e = 1;
      }
      if (has[0] && has[1]) {
        const float lap = (dn[0] + dn[1]) - 2.0f * d;
        if (fabsf(lap) > p.depth_rel * d) e = 1;
      }
      if (has[2] && has[3]) {
        const float lap = (dn[2] + dn[3]) - 2.0f * d;
        if (fabsf(lap) > p.depth_rel * d) e = 1;
      }
    }
    store_edge(p, E, x, y, valid, e != 0);
  }
}

// ---- TMA-staged edge detection (SSAO, SSGI)
constexpr int ETW = 32, ETH = 16, ESTAGES = 2, ETHREADS = 256;
static_assert(ETH % (2 * (ETHREADS / 32)) == 0, "whole pixel pairs per warp");
constexpr int DOFF = 4, DW = ETW + 2 * DOFF;             // depth staged from x0 - 4 (16-byte start)
constexpr uint32_t DBYTES = DW * (ETH + 2) * 4;          // 2880
template <typename NT> struct EdgeTma;
template <> struct EdgeTma<float4> {
  static constexpr int NOFF = 1, NW = ETW + 2;           // normals staged from x0 - 1
  static constexpr uint32_t NBYTES = NW * (ETH + 2) * 16;
};
template <> struct EdgeTma<half4> {
  static constexpr int NOFF = 2, NW = ETW + 4;           // from x0 - 2 (16-byte start)
  static constexpr uint32_t NBYTES = NW * (ETH + 2) * 8;
};
constexpr uint32_t pad128(uint32_t b) { return (b + 127u) / 128u * 128u; }
template <typename NT> constexpr uint32_t stage_bytes() { return pad128(EdgeTma<NT>::NBYTES) + pad128(DBYTES); }
template <typename NT> constexpr uint32_t edges_tma_smem() { return ESTAGES * stage_bytes<NT>() + 64 + 128; }

__device__ __forceinline__ float3 smem_normal(const float4* s, int i) {
  const float4 v = s[i];
  return make_float3(v.x, v.y, v.z);
}
__device__ __forceinline__ float3 smem_normal(const half4* s, int i) {
  const uint2 raw = reinterpret_cast<const uint2*>(s)[i];
  const __half2 xy = *reinterpret_cast<const __half2*>(&raw.x);
  const __half2 zw = *reinterpret_cast<const __half2*>(&raw.y);
  return make_float3(__low2float(xy), __high2float(xy), __low2float(zw));
}

// One-sample hard shadows of Sec. 3.1 as bits (bit b of word w of a row = pixel 32 w + b;
// 1 lit, 0 shadowed; sky, pixels not beyond the light's near plane or off the map, and
// columns past the image 1): the first pass of soft-shadow edge detection when the frame's
// rows allow TMA.  A CTA covers 32 x 32 pixels, a lane SB_ROWS of them (rows ty + 8 k);
// each step -- depth reads, light-space projections, shadow-map reads -- is issued for all
// of the lane's pixels before the next, so a lane waits on two load latencies in all.
constexpr int SB_ROWS = 4;
template <typename SMT>
__global__ void __launch_bounds__(TX* TY) shadow_bits_kernel(EdgeParams p, const float* __restrict__ depth,
                                                              const SMT* __restrict__ smap) {
  const int W = p.v.W, H = p.v.H;
  const int x = blockIdx.x * TX + threadIdx.x;
  float d[SB_ROWS];
  bool in[SB_ROWS];
#pragma unroll
  for (int k = 0; k < SB_ROWS; ++k) {
    const int y = (blockIdx.y * SB_ROWS + k) * TY + threadIdx.y;
    in[k] = x < W && y < H;
    d[k] = __ldg(depth + (in[k] ? (size_t)y * W + x : 0));
  }
  bool look[SB_ROWS];
  size_t si[SB_ROWS];
  float zl[SB_ROWS];
#pragma unroll
  for (int k = 0; k < SB_ROWS; ++k) {
    const int y = (blockIdx.y * SB_ROWS + k) * TY + threadIdx.y;
    look[k] = false;
    si[k] = 0;
    zl[k] = 0.0f;
    float zr, Xt, Yt;
    if (in[k] && d[k] < p.v.farp && light_coords(p.v, p.L, x, y, d[k], zr, Xt, Yt)) {
      const float S = (float)p.L.S;
      if (Xt >= 0.0f && Xt < S && Yt >= 0.0f && Yt < S) {
        look[k] = true;
        si[k] = (size_t)(int)Yt * p.L.S + (int)Xt;
        zl[k] = zr - p.shadow_bias;
      }
    }
  }
  float z[SB_ROWS];
#pragma unroll
  for (int k = 0; k < SB_ROWS; ++k) z[k] = load_sm(smap, si[k]);
#pragma unroll
  for (int k = 0; k < SB_ROWS; ++k) {
    const int y = (blockIdx.y * SB_ROWS + k) * TY + threadIdx.y;
    // hard_shadow's decision: lit unless projected onto the map and behind its depth
    const bool lit = !look[k] || z[k] >= zl[k];
    const uint32_t b = __ballot_sync(0xffffffffu, lit);
    if (threadIdx.x == 0 && y < H) p.sbits[(size_t)y * p.ewords + blockIdx.x] = b;
  }
}

// SSM: the edge tests also compare each pixel's hard shadow with its in-image neighbours'
// (from p.sbits, written by shadow_bits_kernel).
template <typename NT, bool SSM, bool SCALAR = false>
__global__ void __launch_bounds__(ETHREADS) edges_tma_kernel(const __grid_constant__ CUtensorMap tm_n,
                                                             const __grid_constant__ CUtensorMap tm_d, EdgeParams p,
                                                             uint8_t* __restrict__ E) {
  using T = EdgeTma<NT>;
  constexpr uint32_t NP = pad128(T::NBYTES), SB = stage_bytes<NT>();
  extern __shared__ unsigned char edges_dsm[];
  unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(edges_dsm) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(sbase + ESTAGES * SB);
  zero_words(p);
  const int W = p.v.W, H = p.v.H;
  const int gx = (W + ETW - 1) / ETW, gy = (H + ETH - 1) / ETH;
  const int ntiles = gx * gy;
  const int nlocal = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ESTAGES; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: start the loads of the k-th tile of this CTA into stage k % ESTAGES.  The
  // normals are read once per frame here, while the shading launch later gathers the depth
  // again: their lines are marked first to be evicted from L2, so that the depth rather
  // than the normals is what L2 still holds when the shading launch runs.
  auto issue = [&](int k) {
    const int s = k % ESTAGES;
    const int t = (int)blockIdx.x + k * (int)gridDim.x;
    const int x0 = (t % gx) * ETW, y0 = (t / gx) * ETH;
    unsigned char* st = sbase + s * SB;
    mbar_arrive_expect_tx(&full[s], T::NBYTES + DBYTES);
    tma_load_2d_hint(st, &tm_n, &full[s], (x0 - T::NOFF) * 4, y0 - 1, l2_evict_first_policy());
    tma_load_2d(st + NP, &tm_d, &full[s], x0 - DOFF, y0 - 1);
  };
  if (threadIdx.x == 0)
    for (int k = 0; k < min(ESTAGES, nlocal); ++k) issue(k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float farp = p.v.farp;
  int k = 0;
  bool ok = true;
  for (; k < nlocal; ++k) {
    const int s = k % ESTAGES;
    // warp-uniform: the bit-packed store below is a whole-warp ballot
    ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)(k / ESTAGES) & 1u));
    if (ok) {
      const int t = (int)blockIdx.x + k * (int)gridDim.x;
      const int x0 = (t % gx) * ETW, y0 = (t / gx) * ETH;
      const NT* sn = reinterpret_cast<const NT*>(sbase + s * SB);
      const float* sd = reinterpret_cast<const float*>(sbase + s * SB + NP);
#pragma unroll
      for (int pr = 0; pr < ETH / (2 * (ETHREADS / 32)); ++pr) {
      // the lane's two vertically adjacent pixels (rows r0, r0 + 1 of the tile)
      const int r0 = 2 * warp + 2 * (ETHREADS / 32) * pr, x = x0 + lane, y = y0 + r0;
      const int ly = r0 + 1, cd = lane + DOFF, cn = lane + T::NOFF;
      const float d0 = sd[ly * DW + cd], d1 = sd[(ly + 1) * DW + cd];
      // sky pixels are never edges: with soft shadows, whose tests also read the hard-shadow
      // bits, a warp whose 64 pixels are all sky stores its two zero words without them (3-6
      // us per 1440p frame; for the lighter SSAO/SSGI tests the vote costs more than it saves)
      if constexpr (SSM) {
        if (__all_sync(0xffffffffu, (d0 >= farp) & (d1 >= farp))) {
          store_edge(p, E, x, y, x < W && y < H, false);
          store_edge(p, E, x, y + 1, x < W && y + 1 < H, false);
          continue;
        }
      }
      const float du = sd[(ly - 1) * DW + cd], dd = sd[(ly + 2) * DW + cd];
      const float dl0 = sd[ly * DW + cd - 1], dr0 = sd[ly * DW + cd + 1];
      const float dl1 = sd[(ly + 1) * DW + cd - 1], dr1 = sd[(ly + 1) * DW + cd + 1];
      const float3 nu = smem_normal(sn, (ly - 1) * T::NW + cn), n0 = smem_normal(sn, ly * T::NW + cn);
      const float3 n1 = smem_normal(sn, (ly + 1) * T::NW + cn), nd = smem_normal(sn, (ly + 2) * T::NW + cn);
      const float3 nl0 = smem_normal(sn, ly * T::NW + cn - 1), nr0 = smem_normal(sn, ly * T::NW + cn + 1);
      const float3 nl1 = smem_normal(sn, (ly + 1) * T::NW + cn - 1), nr1 = smem_normal(sn, (ly + 1) * T::NW + cn + 1);
      // The neighbour tests, in one of two forms that compute the same bits: scalar FP32
      // (SCALAR: 32 registers, so 8 CTAs fill every warp slot of the SM -- the faster form
      // for a frame rendered alone with FP32 normals) or packed FP32x2 (more registers,
      // fewer CTAs per SM -- faster for soft shadows and FP16 normals, and for batched or
      // served frames, whose kernels share the SMs with other streams' kernels).
      const float cosT = p.normal_cos, farp2 = farp;
      const bool hasl = x > 0, hasr = x < W - 1;
      const bool hasu0 = y > 0, hasd0 = y + 1 < H, hasd1 = y + 1 < H - 1;
      bool e0, e1;
      if constexpr (SCALAR) {
        // n_p . n_q in the order x, y, z, one IEEE operation each
        auto dot = [](float3 a, float3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; };
        const float hl0 = dot(n0, nl0), hl1 = dot(n1, nl1), hr0 = dot(n0, nr0), hr1 = dot(n1, nr1);
        const float vu0 = dot(n0, nu), vu1 = dot(n1, n0), vd0 = dot(n0, n1), vd1 = dot(n1, nd);
        const float m2d0 = -2.0f * d0, m2d1 = -2.0f * d1;
        const float lapx0 = (dl0 + dr0) + m2d0, lapx1 = (dl1 + dr1) + m2d1;
        const float lapy0 = (du + d1) + m2d0, lapy1 = (d0 + dd) + m2d1;
        const float thr0 = p.depth_rel * d0, thr1 = p.depth_rel * d1;
        e0 = (hasl & ((dl0 >= farp2) | (hl0 < cosT))) | (hasr & ((dr0 >= farp2) | (hr0 < cosT))) |
             (hasu0 & ((du >= farp2) | (vu0 < cosT))) | (hasd0 & ((d1 >= farp2) | (vd0 < cosT))) |
             (hasl & hasr & (fabsf(lapx0) > thr0)) | (hasu0 & hasd0 & (fabsf(lapy0) > thr0));
        e1 = (hasl & ((dl1 >= farp2) | (hl1 < cosT))) | (hasr & ((dr1 >= farp2) | (hr1 < cosT))) |
             ((d0 >= farp2) | (vu1 < cosT)) | (hasd1 & ((dd >= farp2) | (vd1 < cosT))) |
             (hasl & hasr & (fabsf(lapx1) > thr1)) | (hasd1 & (fabsf(lapy1) > thr1));
      } else {
        // n_p . n_q for both pixels at once (two independent IEEE products and sums in the
        // order x, y, z -- the same bits as the scalar expression, products commuting)
        const float2 N0x = make_float2(n0.x, n1.x), N0y = make_float2(n0.y, n1.y), N0z = make_float2(n0.z, n1.z);
        auto dot2 = [&](float3 a, float3 b) {
          const float2 px = __fmul2_rn(N0x, make_float2(a.x, b.x));
          const float2 py = __fmul2_rn(N0y, make_float2(a.y, b.y));
          const float2 pz = __fmul2_rn(N0z, make_float2(a.z, b.z));
          return __fadd2_rn(__fadd2_rn(px, py), pz);
        };
        const float2 hl = dot2(nl0, nl1), hr = dot2(nr0, nr1), vu = dot2(nu, n0), vd = dot2(n1, nd);
        // Laplacians along x for both rows and along y
        // a - b is a + (-b) exactly; -2 d is exact
        const float2 m2d = __fmul2_rn(make_float2(-2.0f, -2.0f), make_float2(d0, d1));
        const float2 lapx = __fadd2_rn(__fadd2_rn(make_float2(dl0, dl1), make_float2(dr0, dr1)), m2d);
        const float2 lapy = __fadd2_rn(__fadd2_rn(make_float2(du, d0), make_float2(d1, dd)), m2d);
        const float2 thr = __fmul2_rn(make_float2(p.depth_rel, p.depth_rel), make_float2(d0, d1));
        // The decisions combine with non-short-circuit & and | (every operand is already in
        // a register, so nothing is saved by skipping one): branch-free predicate logic.
        // pixel 0: up neighbour row r0 - 1, down neighbour pixel 1
        e0 = (hasl & ((dl0 >= farp2) | (hl.x < cosT))) | (hasr & ((dr0 >= farp2) | (hr.x < cosT))) |
             (hasu0 & ((du >= farp2) | (vu.x < cosT))) | (hasd0 & ((d1 >= farp2) | (vd.x < cosT))) |
             (hasl & hasr & (fabsf(lapx.x) > thr.x)) | (hasu0 & hasd0 & (fabsf(lapy.x) > thr.x));
        // pixel 1: up neighbour pixel 0, down neighbour row r0 + 2
        e1 = (hasl & ((dl1 >= farp2) | (hl.y < cosT))) | (hasr & ((dr1 >= farp2) | (hr.y < cosT))) |
             ((d0 >= farp2) | (vu.y < cosT)) | (hasd1 & ((dd >= farp2) | (vd.y < cosT))) |
             (hasl & hasr & (fabsf(lapx.y) > thr.y)) | (hasd1 & (fabsf(lapy.y) > thr.y));
      }
      if constexpr (SSM) {
        // hard-shadow bits of rows y - 1 .. y + 2 (clamped; the has flags drop rows and
        // columns outside the image), the words left and right of the tile's word
        const int wc = x0 >> 5;
        uint32_t sc[4], sl[4], sr[4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const uint32_t* row = p.sbits + (size_t)min(max(y - 1 + rr, 0), H - 1) * p.ewords;
          const uint32_t wl = __ldg(row + max(wc - 1, 0)), wm = __ldg(row + wc),
                         wr = __ldg(row + min(wc + 1, p.ewords - 1));
          sc[rr] = (wm >> lane) & 1u;
          sl[rr] = (__funnelshift_l(wl, wm, 1) >> lane) & 1u;  // pixel x - 1
          sr[rr] = (__funnelshift_r(wm, wr, 1) >> lane) & 1u;  // pixel x + 1
        }
        // pixel 0 in row 1 of the four, pixel 1 in row 2
        const uint32_t s0 = sc[1], s1 = sc[2];
        e0 = e0 | (hasl & (sl[1] != s0)) | (hasr & (sr[1] != s0)) | (hasu0 & (sc[0] != s0)) | (hasd0 & (s1 != s0));
        e1 = e1 | (hasl & (sl[2] != s1)) | (hasr & (sr[2] != s1)) | (s0 != s1) | (hasd1 & (sc[3] != s1));
      }
      e0 = e0 & (d0 < farp2);
      e1 = e1 & (d1 < farp2);
      store_edge(p, E, x, y, x < W && y < H, e0);
      store_edge(p, E, x, y + 1, x < W && y + 1 < H, e1);
      }
    }
    // every thread is done with stage s before it is refilled; a failed wait anywhere
    // ends the CTA's walk
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0 && k + ESTAGES < nlocal) issue(k + ESTAGES);
  }
  if (!ok && threadIdx.x == 0) {
    atomicOr(p.fault, FAULT_EDGES_WAIT);
    // the loads of tiles k .. k + ESTAGES - 1 may still be in flight: let them land
    // (again with a limit) before the CTA's shared memory is released
    for (int j = k; j < min(k + ESTAGES, nlocal); ++j) mbar_wait(&full[j % ESTAGES], (uint32_t)(j / ESTAGES) & 1u);
  }
}

template <typename NT, bool SSM, bool SCALAR = false>
int edges_tma_grid() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(edges_tma_kernel<NT, SSM, SCALAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)edges_tma_smem<NT>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edges_tma_kernel<NT, SSM, SCALAR>, ETHREADS,
                                                  edges_tma_smem<NT>());
    blocks = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  }
  return blocks;
}

// Tensor maps of the frame's normals and depth for the TMA kernel; false when the frame's
// layout does not allow TMA (rows not a multiple of 16 bytes, unaligned base).
template <typename NT>
bool edge_maps(const EdgeParams& p, const float* depth, const void* normal, CUtensorMap* tn, CUtensorMap* td) {
  const int W = p.v.W, H = p.v.H;
  if (W % 4 != 0 || (reinterpret_cast<uintptr_t>(depth) & 15) || (reinterpret_cast<uintptr_t>(normal) & 15))
    return false;
  using T = EdgeTma<NT>;
  // normals as a plane of 4 W scalars per row, so that one box row is 4 NW contiguous scalars
  const uint64_t dims[2] = {4 * (uint64_t)W, (uint64_t)H}, strides[1] = {(uint64_t)W * sizeof(NT)};
  const uint32_t box[2] = {4 * (uint32_t)T::NW, ETH + 2};
  const bool ok = encode_tensor_map(tn, sizeof(NT) == 16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                    2, normal, dims, strides, box);
  const uint64_t ddims[2] = {(uint64_t)W, (uint64_t)H}, dstrides[1] = {(uint64_t)W * 4};
  const uint32_t dbox[2] = {DW, ETH + 2};
  return ok && encode_tensor_map(td, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, depth, ddims, dstrides, dbox);
}

// The TMA path: false (nothing launched) when the frame's layout does not allow it.  For
// soft shadows (SMT: the shadow map's storage) the hard-shadow bits are written first.
template <typename NT, typename SMT = void, bool SCALAR = false>
bool launch_edges_tma(const EdgeParams& p, const float* depth, const void* normal, const void* smap, uint8_t* E,
                      cudaStream_t s) {
  constexpr bool SSM = !std::is_void<SMT>::value;
  CUtensorMap tn, td;
  if (!p.fault || !edge_maps<NT>(p, depth, normal, &tn, &td)) return false;
  if constexpr (SSM) {
    dim3 block(TX, TY), grid((p.v.W + TX - 1) / TX, (p.v.H + TY * SB_ROWS - 1) / (TY * SB_ROWS));
    shadow_bits_kernel<SMT><<<grid, block, 0, s>>>(p, depth, (const SMT*)smap);
    count_launches(1);
  }
  const int tiles = ((p.v.W + ETW - 1) / ETW) * ((p.v.H + ETH - 1) / ETH);
  const int grid = min(tiles, edges_tma_grid<NT, SSM, SCALAR>());
  edges_tma_kernel<NT, SSM, SCALAR><<<grid, ETHREADS, edges_tma_smem<NT>(), s>>>(tn, td, p, E);
  return true;
}

}  // namespace

// The bounded-wait self-check: one thread arms an mbarrier phase that expects 16 bytes of
// transactions which no copy will ever bring, then waits for it exactly as the edge
// kernel waits for its tiles.  The wait gives up after WAIT_CYCLES (about a second) and
// the kernel records FAULT_CHECK_WAIT and returns; nothing faults and nothing hangs.
__global__ void check_wait_kernel(uint32_t* fault) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_arrive_expect_tx(&bar, 16u);
    if (!mbar_wait(&bar, 0u)) atomicOr(fault, FAULT_CHECK_WAIT);
  }
}

cudaError_t launch_check_wait(uint32_t* fault, cudaStream_t s) {
  check_wait_kernel<<<1, 32, 0, s>>>(fault);
  count_launches(1);
  return cudaGetLastError();
}

void edges_prepare() {
  edges_tma_grid<float4, false, true>();
  edges_tma_grid<float4, false>();
  edges_tma_grid<half4, false>();
  edges_tma_grid<float4, true>();
  edges_tma_grid<half4, true>();
}

cudaError_t launch_edges(const EdgeParams& p, const float* depth, const void* normal, int half_normal,
                         const float* smap, uint8_t* E, cudaStream_t s) {
  dim3 block(TX, TY), grid((p.v.W + TX - 1) / TX, (p.v.H + TY - 1) / TY);
  if (!p.ssm) {
    const bool tma = half_normal   ? launch_edges_tma<half4>(p, depth, normal, nullptr, E, s)
                     : p.concurrent ? launch_edges_tma<float4>(p, depth, normal, nullptr, E, s)
                                    : launch_edges_tma<float4, void, true>(p, depth, normal, nullptr, E, s);
    if (!tma) {
      dim3 dgrid((p.v.W + TX - 1) / TX, (p.v.H + TY * ER - 1) / (TY * ER));
      if (half_normal) edges_direct_kernel<half4><<<dgrid, block, 0, s>>>(p, depth, (const half4*)normal, E);
      else edges_direct_kernel<float4><<<dgrid, block, 0, s>>>(p, depth, (const float4*)normal, E);
    }
  } else if (p.sbits && (half_normal ? launch_edges_tma<half4, float>(p, depth, normal, smap, E, s)
                                     : launch_edges_tma<float4, float>(p, depth, normal, smap, E, s))) {
    // soft shadows, two passes: shadow bits, then the TMA edge kernel
  } else if (half_normal) {
    edges_kernel<half4, float><<<grid, block, 0, s>>>(p, depth, (const half4*)normal, smap, E);
  } else {
    edges_kernel<float4, float><<<grid, block, 0, s>>>(p, depth, (const float4*)normal, smap, E);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr

namespace mrr {

bool encode_tensor_map(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* base,
                       const uint64_t* dims, const uint64_t* strides, const uint32_t* box) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  if (!encode || rank < 1 || rank > 5) return false;
  cuuint64_t gd[5], gs[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
  }
  for (int i = 0; i + 1 < rank; ++i) gs[i] = strides[i];
  return encode(map, type, (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace mrr
