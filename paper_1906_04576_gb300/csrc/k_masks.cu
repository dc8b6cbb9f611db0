// k_masks.cu -- the per-level masks of Sec. 3.1 / Table 1, the stencil of Sec. 4.1 and
// the dense work lists that replace the stencil test on the GPU.
//
// masks_kernel: ONE launch computes every level.  A CTA owns a 32x32 full-resolution
//   tile (16x16 at level 1, 8x8 at level 2, ...) and stages the edge image of the tile
//   plus a 24-pixel halo in shared memory once.  For each blurred level i it forms the
//   downsampled edge image D_i (block maximum) over the tile and an R_i halo, blurs it
//   horizontally then vertically (taps in ascending order, one fused multiply-add each,
//   the Gaussian held in registers), sets S_i = [a_i > 0] OR-ed with the set texels of
//   the previous enabled finer level inside the block (inclusive nesting, Fig. 2/3 --
//   the children of a texel always lie in the same tile), and writes a_i, S_i.  The
//   coarsest level is written as a = 1, S = 1; disabled levels as 0.  Finally every
//   pixel's owning level (the finest enabled level whose stencil covers it).
// compact_count_kernel / compact_scatter_kernel: deterministic stream compaction of
//   every level's stencil into a row-major list of (y << 16) | x.  Pass 1 counts the set
//   texels of each 4096-texel chunk; pass 2 gives each chunk its exclusive prefix (a
//   block reduction over the preceding chunk counts of its level); every lane loads its 16
//   texels at once, and a warp shuffle scan plus the per-warp totals give each lane its
//   output position, so list order = index order and no warp of the shading kernel idles
//   on an unmasked texel.
#include "mrr_internal.cuh"

namespace mrr {

namespace {

constexpr int TS = MASK_TILE;            // 32
constexpr int MG = MASK_MARGIN;          // 24
constexpr int ES = TS + 2 * MG;          // 80: staged edge image side
constexpr int MAXR = 6;
constexpr int DMAX = TS + 2 * MAXR;      // 44: largest D region side (level 0)
constexpr int MTHREADS = 256;            // as 32 x 8
constexpr int S_TOTAL = TS * TS + (TS / 2) * (TS / 2) + (TS / 4) * (TS / 4) + (TS / 8) * (TS / 8);

template <int I> struct LevelShape {  // level I of a tile: side, smem stencil offset
  static constexpr int T = TS >> I;
  static constexpr int OFF = I == 0 ? 0 : LevelShape<I - 1>::OFF + (TS >> (I - 1)) * (TS >> (I - 1));
};
template <> struct LevelShape<-1> {
  static constexpr int T = 0;
  static constexpr int OFF = 0;
};

constexpr int EW = (ES + 31) / 32;      // 32-bit words per staged edge row

struct MaskSmem {
  uint8_t E[ES][ES];
  uint32_t Ebits[ES][EW + 1];           // the same rows as bit masks (one spare word for shifts)
  uint8_t D[DMAX * DMAX];
  float h[DMAX * TS];
  uint8_t S[S_TOTAL];
  float lut[MASK_LUT_MAX];
};

// Bits [c, c + n) of staged edge row r (n <= 32), bit 0 = column c.
__device__ __forceinline__ uint32_t ebits_window(const MaskSmem& sm, int r, int c) {
  const int w = c >> 5, o = c & 31;
  return __funnelshift_r(sm.Ebits[r][w], sm.Ebits[r][w + 1], o);
}

// Level I with blur radius R (both compile-time): D over the tile + R halo, the two
// blur passes, the stencil with nesting from level P (P < 0: none), and the stores.
template <int I, int R, int P>
__device__ __forceinline__ void blur_level(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  constexpr int Ti = LevelShape<I>::T, DN = Ti + 2 * R, BS = 1 << I;
  const int tid = threadIdx.x;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const int Wi = m.Wi[I], Hi = m.Hi[I];
  float g[2 * R + 1];
#pragma unroll
  for (int t = 0; t <= 2 * R; ++t) g[t] = m.g[I][t];
  bool blur;
  if (I == 0) {
    // level 0: D is the edge image itself, so each horizontal window is a slice of a
    // staged bit row; the table (or the taps over the window's bits) gives its sum
    int anyh = 0;
    constexpr uint32_t WMASK = (1u << (2 * R + 1)) - 1u;
    const bool use_lut = m.lut0 != nullptr && (1 << (2 * R + 1)) <= MASK_LUT_MAX;
    for (int k = tid; k < DN * Ti; k += MTHREADS) {
      const int r = k / Ti, c = k - r * Ti;
      const uint32_t win = ebits_window(sm, MG - R + r, MG - R + c) & WMASK;
      float s = 0.0f;
      if (use_lut) {
        s = sm.lut[win];
      } else {
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t)
          if ((win >> t) & 1u) s = s + g[t];
      }
      sm.h[k] = s;
      anyh |= win != 0u;
    }
    blur = __syncthreads_or(anyh) != 0;
  } else {
  // D_I over the tile and its R halo; E outside the image is staged as 0
  int anyd = 0;
  for (int k = tid; k < DN * DN; k += MTHREADS) {
    const int r = k / DN, c = k - r * DN;
    const int qx = q0x - R + c, qy = q0y - R + r;
    uint8_t v = 0;
    if (qx >= 0 && qx < Wi && qy >= 0 && qy < Hi) {
      const uint8_t* e = &sm.E[qy * BS - (y0 - MG)][qx * BS - (x0 - MG)];
#pragma unroll
      for (int by = 0; by < BS; ++by)
#pragma unroll
        for (int bx = 0; bx < BS; ++bx) v |= e[by * ES + bx];
    }
    sm.D[k] = v;
    anyd |= v;
  }
  // no edge within reach of the tile: a_I = 0 here and the blur passes add only zeros
  blur = __syncthreads_or(anyd) != 0;
  if (blur) {
  // horizontal pass: with D in {0,1}, fma(g, D, s) is s + g where D is set and s elsewhere
  for (int k = tid; k < DN * Ti; k += MTHREADS) {
    const int r = k / Ti, c = k - r * Ti;
    const uint8_t* d = &sm.D[r * DN + c];
    float s = 0.0f;
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t)
      if (d[t]) s = s + g[t];
    sm.h[k] = s;
  }
  __syncthreads();
  }
  }
  // vertical pass, stencil, nesting, stores
  uint8_t* Si = sm.S + LevelShape<I>::OFF;
  for (int k = tid; k < Ti * Ti; k += MTHREADS) {
    const int r = k / Ti, c = k - r * Ti;
    const int qx = q0x + c, qy = q0y + r;
    float s = 0.0f;
    if (blur) {
#pragma unroll
      for (int t = 0; t <= 2 * R; ++t) s = fmaf(g[t], sm.h[(r + t) * Ti + c], s);
    }
    uint8_t st = s > 0.0f ? 1 : 0;
    if (P >= 0) {
      constexpr int F = P >= 0 ? I - P : 0, TP = P >= 0 ? LevelShape<(P >= 0 ? P : 0)>::T : 1;
      const uint8_t* Sp = sm.S + LevelShape<(P >= 0 ? P : 0)>::OFF + (r << F) * TP + (c << F);
#pragma unroll
      for (int dy = 0; dy < (1 << F); ++dy)
#pragma unroll
        for (int dx = 0; dx < (1 << F); ++dx) st |= Sp[dy * TP + dx];
    }
    const bool inside = qx < Wi && qy < Hi;
    Si[k] = inside ? st : 0;
    if (inside) {
      m.alpha[I][(size_t)qy * Wi + qx] = s;
      m.stencil[I][(size_t)qy * Wi + qx] = st;
    }
  }
  __syncthreads();
}

template <int I, int P>
__device__ __forceinline__ void blur_dispatch(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  switch (m.R[I]) {
    case 1: blur_level<I, 1, P>(m, sm, x0, y0); break;
    case 2: blur_level<I, 2, P>(m, sm, x0, y0); break;
    case 3: blur_level<I, 3, P>(m, sm, x0, y0); break;
    case 4: blur_level<I, 4, P>(m, sm, x0, y0); break;
    case 5: blur_level<I, 5, P>(m, sm, x0, y0); break;
    default: blur_level<I, 6, P>(m, sm, x0, y0); break;
  }
}

// Level I written as a constant (mode 1: a = 1, S = 1; mode 2: a = 0, S = 0).
template <int I>
__device__ __forceinline__ void fill_level(const MaskParams& m, MaskSmem& sm, int x0, int y0, int mode) {
  constexpr int Ti = LevelShape<I>::T;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const float av = mode == 1 ? 1.0f : 0.0f;
  const uint8_t sv = mode == 1 ? 1 : 0;
  uint8_t* Si = sm.S + LevelShape<I>::OFF;
  for (int k = threadIdx.x; k < Ti * Ti; k += MTHREADS) {
    const int r = k / Ti, c = k - r * Ti;
    const int qx = q0x + c, qy = q0y + r;
    const bool inside = qx < m.Wi[I] && qy < m.Hi[I];
    Si[k] = inside ? sv : 0;
    if (inside && m.alpha[I]) {
      m.alpha[I][(size_t)qy * m.Wi[I] + qx] = av;
      m.stencil[I][(size_t)qy * m.Wi[I] + qx] = sv;
    }
  }
  __syncthreads();
}

// Level I, whose previous enabled finer level is P (-1: none).
template <int I, int P>
__device__ __forceinline__ void do_level(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  const int mode = m.mode[I];
  if (mode == 0) blur_dispatch<I, P>(m, sm, x0, y0);
  else fill_level<I>(m, sm, x0, y0, mode);
}

// The levels in order; blurred levels are 0..2 (the coarsest, at most 3, is a fill).
// `prev` tracks the previous enabled level for nesting (disabled levels are skipped).
__device__ __forceinline__ void all_levels(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  do_level<0, -1>(m, sm, x0, y0);
  if (m.L < 2) return;
  const bool en0 = m.mode[0] != 2;
  if (en0) do_level<1, 0>(m, sm, x0, y0);
  else do_level<1, -1>(m, sm, x0, y0);
  if (m.L < 3) return;
  const bool en1 = m.mode[1] != 2;
  if (en1) do_level<2, 1>(m, sm, x0, y0);
  else if (en0) do_level<2, 0>(m, sm, x0, y0);
  else do_level<2, -1>(m, sm, x0, y0);
  if (m.L < 4) return;
  fill_level<3>(m, sm, x0, y0, m.mode[3]);  // level 3 can only be the coarsest
}

__global__ void __launch_bounds__(MTHREADS) masks_kernel(MaskParams m, const uint8_t* __restrict__ E) {
  __shared__ MaskSmem sm;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
  const int W = m.W, H = m.H;
  // stage the edge image of the tile + margin (zero outside the image)
  if ((W & 3) == 0) {
    constexpr int Q = ES / 4;
    for (int k = threadIdx.x; k < ES * Q; k += MTHREADS) {
      const int r = k / Q, c = (k - r * Q) * 4;
      const int y = y0 - MG + r, x = x0 - MG + c;  // x and W multiples of 4: all 4 in or all out
      uchar4 v = make_uchar4(0, 0, 0, 0);
      if (y >= 0 && y < H && x >= 0 && x < W) v = __ldg(reinterpret_cast<const uchar4*>(E + (size_t)y * W + x));
      *reinterpret_cast<uchar4*>(&sm.E[r][c]) = v;
    }
  } else {
    for (int k = threadIdx.x; k < ES * ES; k += MTHREADS) {
      const int r = k / ES, c = k - r * ES;
      const int y = y0 - MG + r, x = x0 - MG + c;
      sm.E[r][c] = (y >= 0 && y < H && x >= 0 && x < W) ? __ldg(E + (size_t)y * W + x) : 0;
    }
  }
  __syncthreads();
  // bit rows of the staged edge image (bit c of word c/32 = column c) and the level-0 table
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < ES; r += MTHREADS / 32) {
#pragma unroll
      for (int w = 0; w <= EW; ++w) {
        const int c = w * 32 + lane;
        const uint32_t b = __ballot_sync(0xffffffffu, c < ES && sm.E[r][c] != 0);
        if (lane == 0) sm.Ebits[r][w] = b;
      }
    }
    if (m.lut0 && m.mode[0] == 0 && (1 << (2 * m.R[0] + 1)) <= MASK_LUT_MAX)
      for (int k = threadIdx.x; k < (1 << (2 * m.R[0] + 1)); k += MTHREADS) sm.lut[k] = __ldg(m.lut0 + k);
  }
  __syncthreads();
  all_levels(m, sm, x0, y0);
  if (m.label) {
    for (int r = ty; r < TS; r += 8) {
      const int y = y0 + r, x = x0 + tx;
      if (y >= H || x >= W) continue;
      uint8_t lab = 0xFF;
#pragma unroll
      for (int i = MRR_MAX_LEVELS - 1; i >= 0; --i) {
        if (i >= m.L || m.mode[i] == 2) continue;
        const int Ti = TS >> i;
        const int off = i == 0 ? 0 : (i == 1 ? LevelShape<1>::OFF : (i == 2 ? LevelShape<2>::OFF : LevelShape<3>::OFF));
        if (sm.S[off + (r >> i) * Ti + (tx >> i)]) lab = (uint8_t)i;
      }
      m.label[(size_t)y * W + x] = lab;
    }
  }
}

// Which level slot does this block serve?
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
#pragma unroll
  for (int w = 0; w < COMPACT_THREADS / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(COMPACT_THREADS) compact_count_kernel(CompactParams p) {
  __shared__ uint32_t red[COMPACT_THREADS / 32];
  const int l = slot_of(p, blockIdx.x);
  const int c = blockIdx.x - p.chunk_begin[l];
  const uint32_t n = (uint32_t)p.Wi[l] * (uint32_t)p.Hi[l];
  const uint8_t* S = p.stencil[l];
  const uint32_t base = (uint32_t)c * COMPACT_CHUNK + threadIdx.x * (COMPACT_CHUNK / COMPACT_THREADS);
  uint32_t cnt = 0;
  if (base + 16 <= n && ((reinterpret_cast<uintptr_t>(S + base) & 15) == 0)) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(S + base));
    cnt = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);  // bytes are 0 or 1
  } else {
    for (uint32_t k = base; k < base + 16 && k < n; ++k) cnt += S[k] ? 1u : 0u;
  }
  const uint32_t tot = block_sum(cnt, red);
  if (threadIdx.x == 0) p.chunk_counts[blockIdx.x] = tot;
  if (blockIdx.x == 0 && threadIdx.x < MRR_MAX_LEVELS && ((p.zero_mask >> threadIdx.x) & 1))
    p.counts[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(COMPACT_THREADS) compact_scatter_kernel(CompactParams p) {
  __shared__ uint32_t red[COMPACT_THREADS / 32];
  __shared__ uint32_t wsum[COMPACT_THREADS / 32];
  const int l = slot_of(p, blockIdx.x);
  const int c0 = p.chunk_begin[l];
  const int c = blockIdx.x - c0;
  const uint32_t Wi = (uint32_t)p.Wi[l];
  const uint32_t n = Wi * (uint32_t)p.Hi[l];
  const uint8_t* S = p.stencil[l];
  // each lane owns 16 consecutive texels, loaded at once (one 16-byte load when aligned)
  constexpr int PER_LANE = COMPACT_CHUNK / COMPACT_THREADS;  // 16
  const uint32_t base = (uint32_t)c * COMPACT_CHUNK + threadIdx.x * PER_LANE;
  uint32_t bits = 0;  // bit b: texel base + b is set
  if (base + PER_LANE <= n && ((reinterpret_cast<uintptr_t>(S + base) & 15) == 0)) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(S + base));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int b = 0; b < PER_LANE; ++b) bits |= ((w[b >> 2] >> (8 * (b & 3))) & 0xFFu) ? (1u << b) : 0u;
  } else {
    for (int b = 0; b < PER_LANE; ++b)
      if (base + b < n && S[base + b]) bits |= 1u << b;
  }
  // exclusive prefix of this chunk within its level (sum of the preceding chunk counts)
  uint32_t part = 0;
  for (int k = c0 + threadIdx.x; k < (int)blockIdx.x; k += COMPACT_THREADS) part += p.chunk_counts[k];
  const uint32_t offset = block_sum(part, red);
  // lane prefix within the warp, then warp prefix within the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t mine = __popc(bits);
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t pos = offset + incl - mine;
  for (int w = 0; w < warp; ++w) pos += wsum[w];
  uint32_t* list = p.list[l];
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    const uint32_t idx = base + b;
    const uint32_t y = idx / Wi, x = idx - y * Wi;
    list[pos++] = (y << 16) | x;
  }
  if (threadIdx.x == COMPACT_THREADS - 1 && (int)blockIdx.x == p.chunk_begin[l + 1] - 1)
    p.counts[p.level_of[l]] = pos;
}

}  // namespace

cudaError_t launch_masks(const MaskParams& m, const uint8_t* E, cudaStream_t s) {
  dim3 grid((m.W + TS - 1) / TS, (m.H + TS - 1) / TS);
  masks_kernel<<<grid, MTHREADS, 0, s>>>(m, E);
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

}  // namespace mrr
