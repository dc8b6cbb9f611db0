// k_masks.cu -- the per-level masks of Sec. 3.1 / Table 1, the stencil of Sec. 4.1 and
// the dense work lists that replace the stencil test on the GPU.
//
// masks_kernel: ONE launch computes every level (and, for a whole frame, the work lists
//   too).  A CTA owns a 32x32 full-resolution tile (16x16 at level 1, 8x8 at level 2, ...)
//   and stages the edge image of the tile plus a 24-pixel halo as bit rows.  Every tap of
//   a truncated Gaussian is positive, so a_i > 0 exactly where the (2R_i+1)^2 window of the
//   downsampled edge image D_i (block maximum) holds an edge: the stencil before nesting
//   is a box dilation, computed on bit rows -- one warp per level (row ORs of shifted
//   words, then column ORs across lanes).  Warp I then ORs into level I the children of
//   the finer enabled levels (inclusive nesting, Fig. 2/3 -- children always lie in the
//   same tile) and, for a whole frame, reserves level I's list room with one atomicAdd.
//   A tile with no edge anywhere in its staged rows (most of a typical frame) has empty
//   masks at every blurred level: it skips the bit phase, and on the frame path writes its
//   constant levels directly.
//   Last, every thread writes its texels: a_i is evaluated only where the dilation is set
//   -- the horizontal sums over the (2R_i+1)-bit windows (a table of the exact window sums
//   where one is given; above level 0 each row's sums are computed once, beside its D row,
//   and shared by the texels of the column), the vertical taps with one fused multiply-add
//   each in ascending order, the definition's arithmetic exactly -- and is 0 elsewhere.  The
//   coarsest level is written as a = 1, S = 1; disabled levels as 0.  On the frame path
//   level 0's a_0 feeds only the level-0 blend's min(w_0 a_0, 1), so within the radius r1
//   of an edge, where that is 1 whatever a_0's exact value (MaskParams::sure0), 1 is
//   written instead.  Staged calls also get every pixel's owning level (the finest enabled
//   level whose stencil covers it).
// compact_count_kernel / compact_scatter_kernel: deterministic stream compaction of
//   every level's stencil into a row-major list of (y << 16) | x.  Pass 1 counts the set
//   texels of each 4096-texel chunk; pass 2 gives each chunk its exclusive prefix (a
//   block reduction over the preceding chunk counts of its level); every lane loads its 16
//   texels at once, and a warp shuffle scan plus the per-warp totals give each lane its
//   output position, so list order = index order and no warp of the shading kernel idles
//   on an unmasked texel.
#include <cmath>
#include <cstring>

#include "mrr_internal.cuh"

namespace mrr {

namespace {

constexpr int TS = MASK_TILE;            // 32: tile side (full-resolution pixels)
constexpr int MG = MASK_MARGIN;          // 24: halo rows above / below the tile
constexpr int ER = TS + 2 * MG;          // 80 staged edge rows
constexpr int EWORDS = 3;                // 96 staged edge columns: [x0 - 32, x0 + 64)
constexpr int EX = 32;                   // column of the tile's first pixel in the staged rows
constexpr int MAXR = 6;
constexpr int MTHREADS = 128;            // threads per CTA
static_assert(ER % (MTHREADS / 32) == 0, "edge rows split evenly over the warps");
static_assert(MTHREADS == 128, "four warps: one per level in the bit phase");

// Horizontal window sums of the blurred levels above 0, column-major: h(t, c) at [c][t],
// t = row of the D region, c = tile column.  The row pitches (34 at level 1, 36 at level 2)
// put a warp's 32 reads of one tap (two rows x 16 columns, four rows x 8 columns) in 32
// different banks.
constexpr int H1P = 34, H2P = 36;

struct MaskSmem {
  uint4 E[ER];                           // edge rows as bits: word w bit b = column 32 w + b (w = 3: zero)
  float H1[TS / 2][H1P];                 // level 1's h(t, c)
  float H2[TS / 4][H2P];                 // level 2's h(t, c)
  uint32_t B[MRR_MAX_LEVELS][TS];        // [a_i > 0] rows (before nesting), tile texels only
  uint32_t S[MRR_MAX_LEVELS][TS];        // stencil rows of every level, tile texels only
  float g[MRR_MAX_LEVELS][16];           // the Gaussians of Table 1
  float lut[MASK_LUT_MAX];
  // frame mode: per-row prefix counts and the tile's first list position per level
  uint32_t rowpre[MRR_MAX_LEVELS][TS];
  uint32_t excl[MRR_MAX_LEVELS];
  // frame mode, level 0: rows of the pixels within r1 of an edge (alpha 1 without a_0),
  // and per warp the pixels whose a_0 is still needed, (row << 5) | column
  uint32_t sure[TS];
  uint16_t ring[MTHREADS / 32][TS * TS / (MTHREADS / 32)];
};

// Sum of the taps g[t] whose bit t is set in win, in ascending t, one rounding per add.
__device__ __forceinline__ float window_sum(uint32_t win, const float* g) {
  float s = 0.0f;
  while (win) {
    const int t = __ffs(win) - 1;
    s = s + g[t];
    win &= win - 1u;
  }
  return s;
}

// One bit per aligned group of G bits: bit j of the result is the OR of bits
// [G j, G j + G) of w.
template <int G>
__device__ __forceinline__ uint32_t group_or(uint32_t w) {
  static_assert(G == 2 || G == 4, "levels 1 and 2");
  uint32_t x;
  if (G == 2) {
    x = (w | (w >> 1)) & 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
  } else {
    x = w | (w >> 1);
    x = (x | (x >> 2)) & 0x11111111u;
    x = (x | (x >> 3)) & 0x03030303u;
    x = (x | (x >> 6)) & 0x000F000Fu;
    x = (x | (x >> 12)) & 0x000000FFu;
  }
  return x;
}

// Row t of D_I over the D region (DN = Ti + 2R texels from level row q0y - R and level
// column q0x - R): the OR of the 2^I staged rows of the block row, each aligned group of
// 2^I bits reduced to one.  Edges outside the image are staged as zeros, so blocks outside
// the level give 0, as the block maximum must.
template <int I, int R>
__device__ __forceinline__ uint32_t d_row(const MaskSmem& sm, int t) {
  constexpr int G = 1 << I, DN = (TS >> I) + 2 * R;
  constexpr int row0 = MG - R * G, col0 = EX - R * G;
  static_assert(row0 >= 0 && col0 >= 0 && col0 % G == 0, "halo inside the staged rows");
  uint4 e = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
  for (int k = 0; k < G; ++k) {
    const uint4 w = sm.E[row0 + t * G + k];
    e.x |= w.x;
    e.y |= w.y;
    e.z |= w.z;
  }
  const unsigned long long full = (unsigned long long)group_or<G>(e.x) |
                                  ((unsigned long long)group_or<G>(e.y) << (32 / G)) |
                                  ((unsigned long long)group_or<G>(e.z) << (64 / G));
  return (uint32_t)(full >> (col0 / G)) & ((1u << DN) - 1u);
}

// Bits of the tile texels of level I that lie inside the level, for tile row r (0: none).
template <int I>
__device__ __forceinline__ uint32_t valid_row(const MaskParams& m, int x0, int y0, int r) {
  constexpr int Ti = TS >> I;
  const int q0x = x0 >> I, q0y = y0 >> I;
  if (r >= Ti || q0y + r >= m.Hi[I]) return 0u;
  const int n = min(Ti, m.Wi[I] - q0x);
  return n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
}

// ---- the stencil before nesting, B_i = [a_i > 0], as bits.  Every tap of the truncated
// Gaussian is positive, so a_i(q) > 0 exactly when the (2R+1) x (2R+1) window of D_i around
// q holds an edge: B_i is the box dilation of D_i (a sum of non-negative terms with a
// positive one stays positive in floating point; the smallest product of two taps is far
// above the underflow threshold).

// Level 0, radius R: lane = tile row.  Row dilation of staged row er: bit c = OR of the
// columns x0 + c - R .. x0 + c + R.
template <int R>
__device__ __forceinline__ uint32_t row_dilate0(const MaskSmem& sm, int er) {
  const uint4 row = sm.E[er];
  const uint32_t lo = __funnelshift_r(row.x, row.y, 32 - R);  // bit k: column x0 - R + k
  const uint32_t hi = __funnelshift_r(row.y, row.z, 32 - R);  // bit k: column x0 + 32 - R + k
  const unsigned long long w = ((unsigned long long)hi << 32) | lo;
  unsigned long long d = 0ull;
#pragma unroll
  for (int t = 0; t <= 2 * R; ++t) d |= w >> t;
  return (uint32_t)d;
}

template <int R>
__device__ __forceinline__ void blur_bits0(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  const int lane = threadIdx.x & 31;
  // dilated rows of tile rows lane - R (a) and 32 + lane - R (b, lanes < 2R)
  const uint32_t a = row_dilate0<R>(sm, MG - R + lane);
  const uint32_t b = lane < 2 * R ? row_dilate0<R>(sm, MG - R + 32 + lane) : 0u;
  uint32_t v = 0u;
#pragma unroll
  for (int t = 0; t <= 2 * R; ++t) {
    const int src = lane + t;
    const uint32_t va = __shfl_sync(0xffffffffu, a, src & 31);
    const uint32_t vb = __shfl_sync(0xffffffffu, b, src & 31);
    v |= src < 32 ? va : vb;
  }
  v &= valid_row<0>(m, x0, y0, lane);
  sm.B[0][lane] = v;
  sm.S[0][lane] = v;
}

// Frame mode, level 0: bit c of sure[lane] is set when an edge pixel lies within
// Chebyshev distance r1 = m.sure0 (0..6) of tile pixel (lane, c) -- the box dilation of the
// staged edge rows, as blur_bits0 computes it for a runtime radius.
__device__ __forceinline__ void sure_bits0(const MaskParams& m, MaskSmem& sm) {
  const int lane = threadIdx.x & 31;
  const int r1 = m.sure0;
  auto rowd = [&](int er) {
    const uint4 row = sm.E[er];
    // clamped funnel shifts: r1 = 0 shifts by 32
    const uint32_t lo = __funnelshift_rc(row.x, row.y, 32 - r1);  // bit k: column x0 - r1 + k
    const uint32_t hi = __funnelshift_rc(row.y, row.z, 32 - r1);  // bit k: column x0 + 32 - r1 + k
    const unsigned long long w = ((unsigned long long)hi << 32) | lo;
    unsigned long long d = 0ull;
    for (int t = 0; t <= 2 * r1; ++t) d |= w >> t;
    return (uint32_t)d;
  };
  const uint32_t a = rowd(MG - r1 + lane);
  const uint32_t b = lane < 2 * r1 ? rowd(MG - r1 + 32 + lane) : 0u;
  uint32_t v = 0u;
  for (int t = 0; t <= 2 * r1; ++t) {
    const int src = lane + t;
    const uint32_t va = __shfl_sync(0xffffffffu, a, src & 31);
    const uint32_t vb = __shfl_sync(0xffffffffu, b, src & 31);
    v |= src < 32 ? va : vb;
  }
  sm.sure[lane] = v;
}

// Level I >= 1, radius R: lane t < DN computes row t of D_I over the blur region (level
// rows q0y - R .. q0y + Ti + R - 1, columns q0x - R ..) and, for every tile column c, the
// horizontal sum h(t, c) of the taps over the set bits of the row's (2R+1)-bit window at c
// (the table of exact window sums where one is given); lane r < Ti the dilation.  The sums
// are shared by the 2R+1 texels of a column that read them.
template <int I, int R>
__device__ __forceinline__ void blur_bits(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  constexpr int Ti = TS >> I, DN = Ti + 2 * R;
  static_assert(DN <= 32, "a D region fits one warp");
  static_assert(I == 1 || I == 2, "blurred levels above 0 are 1 and 2");
  constexpr int HP = I == 1 ? H1P : H2P;
  static_assert(DN <= HP, "a D region fits the pitch");
  constexpr uint32_t WMASK = (1u << (2 * R + 1)) - 1u;
  const int lane = threadIdx.x & 31;
  const uint32_t d = lane < DN ? d_row<I, R>(sm, lane) : 0u;
  if (lane < DN) {
    float* hs = I == 1 ? &sm.H1[0][0] : &sm.H2[0][0];
    const float* lut = m.lut[I];
    // the table's lookups all requested at once; without a table, the sums one by one
    if (lut) {
#pragma unroll
      for (int c = 0; c < Ti; ++c) hs[c * HP + lane] = __ldg(lut + ((d >> c) & WMASK));
    } else {
#pragma unroll 1
      for (int c = 0; c < Ti; ++c) hs[c * HP + lane] = window_sum((d >> c) & WMASK, sm.g[I]);
    }
  }
  uint32_t h = 0u;
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) h |= d >> k;
  h &= Ti >= 32 ? 0xFFFFFFFFu : ((1u << Ti) - 1u);
  uint32_t v = 0u;
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) v |= __shfl_sync(0xffffffffu, h, (lane + k) & 31);
  v &= valid_row<I>(m, x0, y0, lane);
  if (lane < Ti) {
    sm.B[I][lane] = v;
    sm.S[I][lane] = v;
  }
}

// Level I as a constant: mode 1 (a = 1, S = 1) or mode 2 (a = 0, S = 0).
template <int I>
__device__ __forceinline__ void fill_bits(const MaskParams& m, MaskSmem& sm, int x0, int y0, int mode) {
  constexpr int Ti = TS >> I;
  const int lane = threadIdx.x & 31;
  const uint32_t v = mode == 1 ? valid_row<I>(m, x0, y0, lane) : 0u;
  if (lane < Ti) {
    sm.B[I][lane] = v;
    sm.S[I][lane] = v;
  }
}

// One bit per aligned group of G bits (G = 2, 4 or 8).
template <int G>
__device__ __forceinline__ uint32_t group_or_any(uint32_t w) {
  if (G == 8) {
    uint32_t x = w | (w >> 1);
    x |= x >> 2;
    x |= x >> 4;
    x &= 0x01010101u;
    return (x | (x >> 7) | (x >> 14) | (x >> 21)) & 0xFu;
  }
  return group_or<G == 8 ? 2 : G>(w);
}

// Phase 2, warp I: level I's final stencil rows and, in frame mode, its row prefix counts
// and list reservation.  Inclusive nesting (Fig. 2/3) sets S_I where any child in the
// previous enabled finer level is set; that level's stencil holds its own children, so
// nesting composes: S_I = B_I OR, for every finer level P, B_P grouped over level I's
// 2^(I-P) x 2^(I-P) blocks (disabled levels have B = 0).  Every level is thus final
// without waiting for the others, and the four scans and reservations run side by side.
// Lane = tile row of level I.
template <int I>
__device__ __forceinline__ void final_level(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  constexpr int Ti = TS >> I;
  const int lane = threadIdx.x & 31;
  uint32_t s = lane < Ti ? (m.disjoint ? sm.S[I][lane] : sm.B[I][lane]) : 0u;
  if (I > 0 && m.mode[I] == 0 && lane < Ti && !m.disjoint) {
    uint32_t kids = 0u;
#pragma unroll
    for (int P = 0; P < I; ++P) {
      constexpr int FMAX = I;  // F = I - P <= I
      const int F = I - P;
      uint32_t rows = 0u;
#pragma unroll
      for (int j = 0; j < (1 << FMAX); ++j)
        if (j < (1 << F)) rows |= sm.B[P][(lane << F) + j];
      kids |= F == 1 ? group_or_any<2>(rows) : (F == 2 ? group_or_any<4>(rows) : group_or_any<8>(rows));
    }
    s |= kids & valid_row<I>(m, x0, y0, lane);
    sm.S[I][lane] = s;
  }
  if (!m.a0c || m.mode[I] == 2) return;
  // frame mode: each tile reserves room for its set texels of the level with one atomicAdd
  // on the level's count (zero before the launch); the entries go there in tile-local
  // row-major order.  The order of the tiles within a list is whatever order the tiles
  // reached their atomics; shading never depends on it (every entry is shaded and stored
  // on its own), and the count is exact.
  const uint32_t pc = (uint32_t)__popc(s);
  uint32_t inc = pc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane < Ti) sm.rowpre[I][lane] = inc - pc;
  const uint32_t cnt = __shfl_sync(0xffffffffu, inc, 31);
  if (lane == 0) sm.excl[I] = cnt ? atomicAdd(m.counts + I, cnt) : 0u;
}

// The disjoint-tile ablation (the variant Sec. 3.1 rejects), warp 0: level I keeps only the
// blocks of its own mask of which no finer enabled level renders any pixel -- every finer
// level's final stencil grouped to level I's texels and removed -- coarser levels after
// finer ones.  Lane = tile row.
__device__ __forceinline__ void disjoint_bits(const MaskParams& m, MaskSmem& sm) {
  const int lane = threadIdx.x & 31;
  for (int I = 1; I < m.L; ++I) {
    const int Ti = TS >> I;
    if (lane < Ti) {
      uint32_t covered = 0u;
      for (int P = 0; P < I; ++P) {
        const int F = I - P;
        uint32_t rows = 0u;
        for (int j = 0; j < (1 << F); ++j) rows |= sm.S[P][(lane << F) + j];
        covered |= F == 1 ? group_or_any<2>(rows) : (F == 2 ? group_or_any<4>(rows) : group_or_any<8>(rows));
      }
      sm.S[I][lane] = sm.B[I][lane] & ~covered;
    }
    __syncwarp();
  }
}

// ---- a_i at one texel, from the same horizontal sums and the same fused multiply-adds
// in ascending tap order as the definition: h(t) = the ascending sum of the taps over the
// set bits of the (2R+1)-bit window (a table of the exact window sums where one is given),
// a = fma(g_2R, h(2R), ... fma(g_0, h(0), 0)).  The vertical taps g_t come straight from the
// kernel's parameters (constant operands once the loop is unrolled), not from shared memory.

// Level 0, tile texel (r, c): windows from the staged edge rows.
template <int R>
__device__ __forceinline__ float alpha0_at(const MaskParams& m, const MaskSmem& sm, bool use_lut, int r, int c) {
  constexpr uint32_t WMASK = (1u << (2 * R + 1)) - 1u;
  const int b = EX - R + c;  // first staged column of the texel's window
  const int k = b >> 5, sh = b & 31;
  auto win_at = [&](int t) {
    const uint4 row = sm.E[MG + r - R + t];
    const uint32_t lo = k == 0 ? row.x : row.y, hi = k == 0 ? row.y : row.z;
    return __funnelshift_r(lo, hi, sh) & WMASK;
  };
  float s = 0.0f;
  if (use_lut) {
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t) s = fmaf(m.g[0][t], sm.lut[win_at(t)], s);
  } else {
#pragma unroll 1
    for (int t = 0; t <= 2 * R; ++t) s = fmaf(m.g[0][t], window_sum(win_at(t), sm.g[0]), s);
  }
  return s;
}

// Level I >= 1, tile texel (r, c): the horizontal sums of rows r .. r + 2R of the D region.
template <int I, int R>
__device__ __forceinline__ float alpha_at(const MaskParams& m, const MaskSmem& sm, int r, int c) {
  const float* h = I == 1 ? &sm.H1[c][r] : &sm.H2[c][r];
  float s = 0.0f;
#pragma unroll
  for (int t = 0; t <= 2 * R; ++t) s = fmaf(m.g[I][t], h[t], s);
  return s;
}

// ---- writing the levels

// Level 0 (mode 0 blurred, 1 constant one, 2 disabled).  Frame mode: the tile's level-0
// list entries (tile-local row-major, at the reserved position) and a_0 beside them -- 1
// where an edge lies within r1 (the blend's alpha is 1 there either way), else the exact
// a_0, evaluated for the warp's queued pixels 32 at a time so that no lane idles on a pixel
// that needs none; staged mode: a_0 and S_0 for every pixel of the tile.  Warp w takes tile
// rows w, w + 4, ...
template <int R>
__device__ __forceinline__ void write_level0(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mode = m.mode[0];
  const bool use_lut = m.lut0 != nullptr && (1 << (2 * R + 1)) <= MASK_LUT_MAX;
  const int x = x0 + lane;
  const size_t cap = (size_t)m.Wi[0] * m.Hi[0];
  if (m.a0c) {
    const uint32_t below = (1u << lane) - 1u;
    uint16_t* q = sm.ring[warp];
    int qn = 0;
    for (int r = warp; r < TS; r += MTHREADS / 32) {
      const uint32_t bits = sm.S[0][r];
      if (bits == 0u) continue;
      const uint32_t ring = mode == 0 ? bits & ~(m.sure0 >= 0 ? sm.sure[r] : 0u) : 0u;
      const bool on = (bits >> lane) & 1u, queued = (ring >> lane) & 1u;
      const size_t pos = (size_t)sm.excl[0] + sm.rowpre[0][r] + __popc(bits & below);
      if (on && pos < cap) {
        m.list[0][pos] = ((uint32_t)(y0 + r) << 16) | (uint32_t)x;
        if (!queued) m.a0c[pos] = 1.0f;
      }
      if (queued) q[qn + __popc(ring & below)] = (uint16_t)((r << 5) | lane);
      qn += __popc(ring);
    }
    __syncwarp();
    for (int k = lane; k < qn; k += 32) {
      const int r = q[k] >> 5, c = q[k] & 31;
      const float a = alpha0_at<R>(m, sm, use_lut, r, c);
      const size_t pos = (size_t)sm.excl[0] + sm.rowpre[0][r] + __popc(sm.S[0][r] & ((1u << c) - 1u));
      if (pos < cap) m.a0c[pos] = a;
    }
    return;
  }
  for (int r = warp; r < TS; r += MTHREADS / 32) {
    const int y = y0 + r;
    const uint32_t bits = sm.S[0][r];
    const bool on = (bits >> lane) & 1u;
    if (y >= m.H || x >= m.W || !m.alpha[0]) continue;
    float a = 0.0f;
    if (on) a = mode == 0 ? alpha0_at<R>(m, sm, use_lut, r, lane) : 1.0f;
    m.alpha[0][(size_t)y * m.W + x] = a;
    m.stencil[0][(size_t)y * m.W + x] = on ? 1 : 0;
  }
}

// Level I >= 1 (radius R when blurred): a_I and S_I of every tile texel inside the level,
// and in frame mode the list entries.  Thread k takes texel k of the tile (row-major).
template <int I, int R>
__device__ __forceinline__ void write_level(const MaskParams& m, const MaskSmem& sm, int x0, int y0) {
  constexpr int Ti = TS >> I;
  const int mode = m.mode[I];
  if (mode == 2 && !m.alpha[I]) return;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const int Wi = m.Wi[I], Hi = m.Hi[I];
  for (int k = threadIdx.x; k < Ti * Ti; k += MTHREADS) {
    const int r = k / Ti, c = k - r * Ti;
    const int qx = q0x + c, qy = q0y + r;
    if (qx >= Wi || qy >= Hi) continue;
    const uint32_t srow = sm.S[I][r];
    const bool st = (srow >> c) & 1u;
    float a = 0.0f;
    if (mode == 1) a = 1.0f;
    else if (mode == 0 && ((sm.B[I][r] >> c) & 1u)) a = alpha_at<I, R>(m, sm, r, c);
    const size_t q = (size_t)qy * Wi + qx;
    m.alpha[I][q] = a;
    m.stencil[I][q] = st ? 1 : 0;
    if (m.a0c && st && mode != 2) {
      const size_t pos = (size_t)sm.excl[I] + sm.rowpre[I][r] + __popc(srow & ((1u << c) - 1u));
      if (pos < (size_t)Wi * Hi) m.list[I][pos] = ((uint32_t)qy << 16) | (uint32_t)qx;
    }
  }
}

// ---- per-level dispatch over the radius (the specialised signatures fix them at compile time)

template <int I>
__device__ __forceinline__ void bits_any(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  if (m.mode[I] != 0) {
    fill_bits<I>(m, sm, x0, y0, m.mode[I]);
    return;
  }
  if (I == 0) {
    switch (m.R[0]) {
      case 1: blur_bits0<1>(m, sm, x0, y0); break;
      case 2: blur_bits0<2>(m, sm, x0, y0); break;
      case 3: blur_bits0<3>(m, sm, x0, y0); break;
      case 4: blur_bits0<4>(m, sm, x0, y0); break;
      case 5: blur_bits0<5>(m, sm, x0, y0); break;
      default: blur_bits0<6>(m, sm, x0, y0); break;
    }
    return;
  }
  constexpr int J = I == 0 ? 1 : (I > 2 ? 2 : I);  // blurred levels are 0..2
  switch (m.R[J]) {
    case 1: blur_bits<J, 1>(m, sm, x0, y0); break;
    case 2: blur_bits<J, 2>(m, sm, x0, y0); break;
    case 3: blur_bits<J, 3>(m, sm, x0, y0); break;
    case 4: blur_bits<J, 4>(m, sm, x0, y0); break;
    case 5: blur_bits<J, 5>(m, sm, x0, y0); break;
    default: blur_bits<J, 6>(m, sm, x0, y0); break;
  }
}

template <int I>
__device__ __forceinline__ void write_any(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  if (I == 0) {
    switch (m.mode[0] == 0 ? m.R[0] : 1) {
      case 1: write_level0<1>(m, sm, x0, y0); break;
      case 2: write_level0<2>(m, sm, x0, y0); break;
      case 3: write_level0<3>(m, sm, x0, y0); break;
      case 4: write_level0<4>(m, sm, x0, y0); break;
      case 5: write_level0<5>(m, sm, x0, y0); break;
      default: write_level0<6>(m, sm, x0, y0); break;
    }
    return;
  }
  constexpr int J = I == 0 ? 1 : I;
  if (m.mode[J] != 0) {
    write_level<J, 1>(m, sm, x0, y0);
    return;
  }
  constexpr int K = J > 2 ? 2 : J;  // blurred levels are 0..2
  switch (m.R[K]) {
    case 1: write_level<K, 1>(m, sm, x0, y0); break;
    case 2: write_level<K, 2>(m, sm, x0, y0); break;
    case 3: write_level<K, 3>(m, sm, x0, y0); break;
    case 4: write_level<K, 4>(m, sm, x0, y0); break;
    case 5: write_level<K, 5>(m, sm, x0, y0); break;
    default: write_level<K, 6>(m, sm, x0, y0); break;
  }
}

// ---- frame mode, a tile with no edge in its staged rows: every blurred or disabled level
// is 0 over the tile and the coarsest level is 1, so the tile's outputs are written
// directly -- the same values and list entries (in the same tile-local row-major order)
// as the general path, without its nesting, scans and per-texel tests.

// Level I (blurred or disabled): a = 0 and S = 0 for every tile texel inside the level;
// thread t takes column t mod Ti of rows t / Ti, t / Ti + 128 / Ti, ...
template <int I>
__device__ __forceinline__ void empty_zero_level(const MaskParams& m, int x0, int y0) {
  constexpr int Ti = TS >> I, RS = MTHREADS / Ti;
  static_assert(I >= 1 && MTHREADS % Ti == 0, "levels above 0");
  if (!m.alpha[I]) return;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const int nvx = min(Ti, m.Wi[I] - q0x), nvy = min(Ti, m.Hi[I] - q0y);
  const int c = threadIdx.x & (Ti - 1);
  if (c >= nvx) return;
  for (int r = threadIdx.x / Ti; r < nvy; r += RS) {
    const size_t q = (size_t)(q0y + r) * m.Wi[I] + q0x + c;
    m.alpha[I][q] = 0.0f;
    m.stencil[I][q] = 0;
  }
}

// Level I (the coarsest, a = 1 and S = 1 everywhere), by one warp: the tile's texels and
// their list entries at one reservation.
template <int I>
__device__ __forceinline__ void empty_one_level(const MaskParams& m, int x0, int y0) {
  constexpr int Ti = TS >> I;
  static_assert(I >= 1, "levels above 0");
  const int lane = threadIdx.x & 31;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const int nvx = min(Ti, m.Wi[I] - q0x), nvy = min(Ti, m.Hi[I] - q0y);
  const uint32_t n = (uint32_t)(nvx * nvy);
  uint32_t base = 0u;
  if (m.list[I] && lane == 0 && n) base = atomicAdd(m.counts + I, n);
  base = __shfl_sync(0xffffffffu, base, 0);
  const size_t cap = (size_t)m.Wi[I] * m.Hi[I];
  for (int r = 0; r < nvy; ++r)
    for (int c = lane; c < nvx; c += 32) {
      const int qx = q0x + c, qy = q0y + r;
      const size_t q = (size_t)qy * m.Wi[I] + qx;
      m.alpha[I][q] = 1.0f;
      m.stencil[I][q] = 1;
      const size_t pos = (size_t)base + (size_t)r * nvx + c;
      if (m.list[I] && pos < cap) m.list[I][pos] = ((uint32_t)qy << 16) | (uint32_t)qx;
    }
}

template <int I>
__device__ __forceinline__ void empty_level(const MaskParams& m, int x0, int y0) {
  if (I >= m.L) return;
  if (m.mode[I] == 1) {
    if ((threadIdx.x >> 5) == 3) empty_one_level<I>(m, x0, y0);
  } else {
    empty_zero_level<I>(m, x0, y0);
  }
}

// Level patterns compiled on their own, so that the kernel holds only the code they run:
//   MASK_SIG_T1_4: four levels, levels 0-2 blurred with radii 3, 5, 6 (Table 1's SSAO and
//                  soft-shadow rows, sigma^2 = 0.924, 1.848, 3.696);
//   MASK_SIG_T1_GI: four levels, level 1 disabled, levels 0 and 2 blurred with radius 3
//                  (Table 1's SSGI rows);
//   MASK_SIG_T1_3: three levels, levels 0 and 1 blurred with radii 3 and 5.
enum { MASK_SIG_ANY = 0, MASK_SIG_T1_4 = 1, MASK_SIG_T1_GI = 2, MASK_SIG_T1_3 = 3 };

// Warp I computes level I's [a > 0] rows (levels 0..3 on warps 0..3).
template <int SIG>
__device__ __forceinline__ void level_bits(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  const int warp = threadIdx.x >> 5;
  if constexpr (SIG == MASK_SIG_T1_4) {
    if (warp == 0) blur_bits0<3>(m, sm, x0, y0);
    else if (warp == 1) blur_bits<1, 5>(m, sm, x0, y0);
    else if (warp == 2) blur_bits<2, 6>(m, sm, x0, y0);
    else fill_bits<3>(m, sm, x0, y0, m.mode[3]);
  } else if constexpr (SIG == MASK_SIG_T1_GI) {
    if (warp == 0) blur_bits0<3>(m, sm, x0, y0);
    else if (warp == 1) fill_bits<1>(m, sm, x0, y0, 2);
    else if (warp == 2) blur_bits<2, 3>(m, sm, x0, y0);
    else fill_bits<3>(m, sm, x0, y0, m.mode[3]);
  } else if constexpr (SIG == MASK_SIG_T1_3) {
    if (warp == 0) blur_bits0<3>(m, sm, x0, y0);
    else if (warp == 1) blur_bits<1, 5>(m, sm, x0, y0);
    else if (warp == 2) fill_bits<2>(m, sm, x0, y0, m.mode[2]);
  } else {
    if (warp == 0) bits_any<0>(m, sm, x0, y0);
    else if (warp == 1 && m.L > 1) bits_any<1>(m, sm, x0, y0);
    else if (warp == 2 && m.L > 2) bits_any<2>(m, sm, x0, y0);
    else if (warp == 3 && m.L > 3) fill_bits<3>(m, sm, x0, y0, m.mode[3]);
  }
  // frame mode: warp 3 (otherwise at most filling the coarsest level) also marks where
  // level 0's alpha is 1 without a_0
  if (warp == 3 && m.a0c && m.sure0 >= 0) sure_bits0(m, sm);
}

template <int SIG>
__device__ __forceinline__ void level_values(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  if constexpr (SIG == MASK_SIG_T1_4) {
    write_level0<3>(m, sm, x0, y0);
    write_level<1, 5>(m, sm, x0, y0);
    write_level<2, 6>(m, sm, x0, y0);
    write_level<3, 1>(m, sm, x0, y0);
  } else if constexpr (SIG == MASK_SIG_T1_GI) {
    write_level0<3>(m, sm, x0, y0);
    write_level<1, 1>(m, sm, x0, y0);
    write_level<2, 3>(m, sm, x0, y0);
    write_level<3, 1>(m, sm, x0, y0);
  } else if constexpr (SIG == MASK_SIG_T1_3) {
    write_level0<3>(m, sm, x0, y0);
    write_level<1, 5>(m, sm, x0, y0);
    write_level<2, 1>(m, sm, x0, y0);
  } else {
    write_any<0>(m, sm, x0, y0);
    if (m.L > 1) write_any<1>(m, sm, x0, y0);
    if (m.L > 2) write_any<2>(m, sm, x0, y0);
    if (m.L > 3) write_any<3>(m, sm, x0, y0);
  }
}

template <int SIG>
__global__ void __launch_bounds__(MTHREADS, 2048 / MTHREADS) masks_kernel(MaskParams m, const uint8_t* __restrict__ E) {
  __shared__ MaskSmem sm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = m.W, H = m.H;
  const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS;
  // stage the edge rows y0-24 .. y0+55, columns x0-32 .. x0+63, as bits (zero outside the image)
  uint32_t* Ew = reinterpret_cast<uint32_t*>(sm.E);
  uint32_t seen = 0u;  // OR of the edge bits this thread staged
  if (m.ebits) {
    // bit-packed edge image: the three words of each staged row
    // the thread's two words (and its lookup-table entry below) are all requested before
    // any is stored
    constexpr int NW = ER * EWORDS, RW = (NW + MTHREADS - 1) / MTHREADS;
    uint32_t v[RW];
#pragma unroll
    for (int j = 0; j < RW; ++j) {
      const int k = threadIdx.x + j * MTHREADS;
      const int r = k / EWORDS, w = k - r * EWORDS;
      const int y = y0 - MG + r, wx = (x0 >> 5) - 1 + w;
      v[j] = 0u;
      if (k < NW && y >= 0 && y < H && wx >= 0 && wx < m.ewords) v[j] = __ldg(m.ebits + (size_t)y * m.ewords + wx);
    }
#pragma unroll
    for (int j = 0; j < RW; ++j) {
      const int k = threadIdx.x + j * MTHREADS;
      if (k < NW) Ew[4 * (k / EWORDS) + (k - (k / EWORDS) * EWORDS)] = v[j];
      seen |= v[j];
    }
    if (threadIdx.x < ER) Ew[4 * threadIdx.x + EWORDS] = 0u;
  } else if ((W & 15) == 0 && ((uintptr_t)E & 15) == 0) {
    // 16 pixels per 16-byte load (segments lie wholly inside or outside the image);
    // every load of the CTA is issued before the first is used
    constexpr int SEGS = EWORDS * 2, TASKS = ER * SEGS, ROUNDS = (TASKS + MTHREADS - 1) / MTHREADS;
    constexpr int BATCH = ROUNDS < 2 ? ROUNDS : 2;  // loads in flight per thread
#pragma unroll
    for (int j0 = 0; j0 < ROUNDS; j0 += BATCH) {
      uint4 v[BATCH];
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int k = threadIdx.x + (j0 + j) * MTHREADS;
        const int r = k / SEGS, sg = k - r * SEGS;
        const int y = y0 - MG + r, x = x0 - EX + 16 * sg;
        v[j] = make_uint4(0u, 0u, 0u, 0u);
        if (j0 + j < ROUNDS && k < TASKS && y >= 0 && y < H && x >= 0 && x < W)
          v[j] = __ldg(reinterpret_cast<const uint4*>(E + (size_t)y * W + x));
      }
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const int k = threadIdx.x + (j0 + j) * MTHREADS;
        if (j0 + j >= ROUNDS || k >= TASKS) break;
        const int r = k / SEGS, sg = k - r * SEGS;
        // one bit per nonzero byte: byte flags 0/1 gathered into a nibble by one multiply
        const uint32_t q0 = (__vcmpne4(v[j].x, 0u) & 0x01010101u) * 0x01020408u;
        const uint32_t q1 = (__vcmpne4(v[j].y, 0u) & 0x01010101u) * 0x01020408u;
        const uint32_t q2 = (__vcmpne4(v[j].z, 0u) & 0x01010101u) * 0x01020408u;
        const uint32_t q3 = (__vcmpne4(v[j].w, 0u) & 0x01010101u) * 0x01020408u;
        const uint32_t bits = (q0 >> 24) | ((q1 >> 24) << 4) | ((q2 >> 24) << 8) | ((q3 >> 24) << 12);
        reinterpret_cast<uint16_t*>(Ew + 4 * r)[sg] = (uint16_t)bits;
        seen |= bits;
      }
    }
    if (threadIdx.x < ER) Ew[4 * threadIdx.x + EWORDS] = 0u;
  } else {
#pragma unroll
    for (int j = 0; j < ER / (MTHREADS / 32); ++j) {
      const int r = warp + j * (MTHREADS / 32);
      const int y = y0 - MG + r;
      const bool row_in = y >= 0 && y < H;
#pragma unroll
      for (int w = 0; w < EWORDS; ++w) {
        const int x = x0 - EX + 32 * w + lane;
        const bool e = row_in && x >= 0 && x < W && __ldg(E + (size_t)y * W + x) != 0;
        const uint32_t b = __ballot_sync(0xffffffffu, e);
        if (lane == 0) Ew[4 * r + w] = b;
        seen |= b;
      }
      if (lane == 0) Ew[4 * r + EWORDS] = 0u;
    }
  }
  if (threadIdx.x < MRR_MAX_LEVELS * 16) {
    const int i = threadIdx.x >> 4, t = threadIdx.x & 15;
    sm.g[i][t] = t < 2 * MAXR + 1 ? m.g[i][t] : 0.0f;
  }
  if (m.lut0 && m.mode[0] == 0 && (1 << (2 * m.R[0] + 1)) <= MASK_LUT_MAX)
    for (int k = threadIdx.x; k < (1 << (2 * m.R[0] + 1)); k += MTHREADS) sm.lut[k] = __ldg(m.lut0 + k);
  const bool any_edge = __syncthreads_or(seen != 0u) != 0;
  if (!any_edge && m.a0c && !m.label && !m.disjoint && m.mode[0] != 1) {
    // frame mode, no edge in reach: level 0 has no pixel (nothing to write on the frame
    // path), the others are constant over the tile
    empty_level<1>(m, x0, y0);
    empty_level<2>(m, x0, y0);
    empty_level<3>(m, x0, y0);
    return;
  }
  // 1. [a_i > 0] of every level as bit rows (one warp per level).  With no edge anywhere in
  // the staged rows every blurred level's window sums are 0 (each D row is made of staged
  // rows only), so [a > 0] is empty there and only the constant levels have bits.
  if (any_edge) {
    level_bits<SIG>(m, sm, x0, y0);
  } else if (warp < m.L) {
    if (warp == 0) fill_bits<0>(m, sm, x0, y0, m.mode[0]);
    else if (warp == 1) fill_bits<1>(m, sm, x0, y0, m.mode[1]);
    else if (warp == 2) fill_bits<2>(m, sm, x0, y0, m.mode[2]);
    else fill_bits<3>(m, sm, x0, y0, m.mode[3]);
  }
  __syncthreads();
  if (m.disjoint) {  // the ablation's stencils, finer levels first
    if (warp == 0) disjoint_bits(m, sm);
    __syncthreads();
  }
  // 2. final stencils (inclusive nesting), prefix counts and list reservations (warp I: level I)
  if (warp < m.L) {
    if (warp == 0) final_level<0>(m, sm, x0, y0);
    else if (warp == 1) final_level<1>(m, sm, x0, y0);
    else if (warp == 2) final_level<2>(m, sm, x0, y0);
    else final_level<3>(m, sm, x0, y0);
  }
  __syncthreads();
  // 4. a_i where it is positive, every level's outputs
  level_values<SIG>(m, sm, x0, y0);
  if (m.label) {
    for (int r = warp; r < TS; r += MTHREADS / 32) {
      const int y = y0 + r, x = x0 + lane;
      if (y >= H || x >= W) continue;
      uint8_t lab = 0xFF;
#pragma unroll
      for (int i = MRR_MAX_LEVELS - 1; i >= 0; --i) {
        if (i >= m.L || m.mode[i] == 2) continue;
        if ((sm.S[i][r >> i] >> (lane >> i)) & 1u) lab = (uint8_t)i;
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

// The level pattern of m when it is one of the specialised ones.
int mask_signature(const MaskParams& m) {
  const bool b0 = m.mode[0] == 0 && m.R[0] == 3;
  if (m.L == 4 && b0 && m.mode[1] == 0 && m.R[1] == 5 && m.mode[2] == 0 && m.R[2] == 6) return MASK_SIG_T1_4;
  if (m.L == 4 && b0 && m.mode[1] == 2 && m.mode[2] == 0 && m.R[2] == 3) return MASK_SIG_T1_GI;
  if (m.L == 3 && b0 && m.mode[1] == 0 && m.R[1] == 5) return MASK_SIG_T1_3;
  return MASK_SIG_ANY;
}

int mask_gauss(double sigma2, float* g) {
  if (!(sigma2 > 0.0)) return 0;
  const int R = (int)std::ceil(3.0 * std::sqrt(sigma2));
  if (R > 6) return R;
  double e[16];
  double sum = 0.0;
  for (int k = -R; k <= R; ++k) {
    e[k + R] = std::exp(-(double)(k * k) / (2.0 * sigma2));
    sum += e[k + R];
  }
  for (int k = 0; k <= 2 * R; ++k) g[k] = (float)(e[k] / sum);
  return R;
}

bool mask_level_params(const mrr_config& c, const mrr_levels* lv, MaskParams& m) {
  std::memset(&m, 0, sizeof m);
  m.W = lv->width[0];
  m.H = lv->height[0];
  m.L = c.num_levels;
  for (int i = 0; i < c.num_levels; ++i) {
    if (!c.enabled[i]) {
      m.mode[i] = 2;
    } else if (i == c.num_levels - 1 || (i == 0 && c.force_level0)) {
      m.mode[i] = 1;
    } else {
      m.mode[i] = 0;
      m.R[i] = mask_gauss((double)c.sigma2[i], m.g[i]);
      if (m.R[i] < 1 || m.R[i] > 6) return false;
    }
    m.Wi[i] = lv->width[i];
    m.Hi[i] = lv->height[i];
    m.alpha[i] = lv->alpha[i];
    m.stencil[i] = lv->stencil[i];
  }
  m.label = lv->label;
  m.disjoint = c.disjoint;
  m.sure0 = -1;
  if (m.mode[0] == 0) {
    const int R = m.R[0];
    const float w = c.weight[0];
    for (int r1 = 0; r1 <= R; ++r1) {
      bool all = true;
      for (int dy = -r1; dy <= r1 && all; ++dy)
        for (int dx = -r1; dx <= r1 && all; ++dx) {
          const float prod = m.g[0][R + dy] * m.g[0][R + dx];
          all = w * prod >= 1.0f;
        }
      if (!all) break;
      m.sure0 = r1;
    }
  }
  return true;
}

cudaError_t launch_masks(const MaskParams& m, const uint8_t* E, cudaStream_t s) {
  dim3 grid((m.W + TS - 1) / TS, (m.H + TS - 1) / TS);
  switch (mask_signature(m)) {
    case MASK_SIG_T1_4: masks_kernel<MASK_SIG_T1_4><<<grid, MTHREADS, 0, s>>>(m, E); break;
    case MASK_SIG_T1_GI: masks_kernel<MASK_SIG_T1_GI><<<grid, MTHREADS, 0, s>>>(m, E); break;
    case MASK_SIG_T1_3: masks_kernel<MASK_SIG_T1_3><<<grid, MTHREADS, 0, s>>>(m, E); break;
    default: masks_kernel<MASK_SIG_ANY><<<grid, MTHREADS, 0, s>>>(m, E); break;
  }
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
