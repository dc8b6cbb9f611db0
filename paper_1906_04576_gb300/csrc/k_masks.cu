// k_masks.cu -- the per-level masks of Sec. 3.1 / Table 1, the stencil of Sec. 4.1 and
// the dense work lists that replace the stencil test on the GPU.
//
// masks_kernel: ONE launch computes every level, bit-parallel (and, for a whole frame,
//   the work lists too -- see frame_lists).  A CTA owns a 32x32
//   full-resolution tile (16x16 at level 1, 8x8 at level 2, ...) and stages the edge
//   image of the tile plus a 24-pixel halo as bit rows (one ballot per 32 pixels).  For
//   each blurred level i it forms the downsampled edge image D_i (block maximum: the OR
//   of 2^i staged rows, each group of 2^i bits OR-ed into one) over the tile and an R_i
//   halo, takes the horizontal blur of every texel from its (2R_i+1)-bit window (at
//   level 0 through a table of the exact window sums), the vertical blur with one fused
//   multiply-add per tap in ascending order, sets S_i = [a_i > 0] OR-ed with its children
//   in the previous enabled finer level (inclusive nesting, Fig. 2/3 -- children always
//   lie in the same tile) and writes a_i, S_i.  The coarsest level is written as a = 1,
//   S = 1; disabled levels as 0.  Finally every pixel's owning level (the finest enabled
//   level whose stencil covers it), read from the stencil bit rows.
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

constexpr int TS = MASK_TILE;            // 32: tile side (full-resolution pixels)
constexpr int MG = MASK_MARGIN;          // 24: halo rows above / below the tile
constexpr int ER = TS + 2 * MG;          // 80 staged edge rows
constexpr int EWORDS = 3;                // 96 staged edge columns: [x0 - 32, x0 + 64)
constexpr int EX = 32;                   // column of the tile's first pixel in the staged rows
constexpr int MAXR = 6;
constexpr int DROWS = TS / 2 + 2 * MAXR; // 28: largest D region side above level 0 (level 1)
constexpr int MTHREADS = 128;            // threads per CTA
constexpr int ROWS0 = TS / (MTHREADS / 32);  // level-0 tile rows per warp
static_assert(ROWS0 % 4 == 0, "level-0 rows come in groups of four");
static_assert(ER % (MTHREADS / 32) == 0, "edge rows split evenly over the warps");
static_assert(DROWS <= 32, "a D row of a level above 0 fits one word");

struct MaskSmem {
  uint4 E[ER];                           // edge rows as bits: word w bit b = column 32 w + b (w = 3: zero)
  uint32_t D[DROWS];                     // D_i rows of the current level >= 1 as bits
  float h[DROWS * TS / 2];               // horizontal pass of the current level >= 1
  float g[MRR_MAX_LEVELS][16];           // the Gaussians of Table 1
  uint32_t S[MRR_MAX_LEVELS][TS];        // stencil rows of every level as bits (tile texels only)
  float lut[MASK_LUT_MAX];
  // frame mode: level 0's a over the tile, per-row prefix counts and the tile's first
  // list position per level
  float a0t[TS][TS];
  uint32_t rowpre[MRR_MAX_LEVELS][TS];
  uint32_t excl[MRR_MAX_LEVELS];
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

// Ballot per-lane stencil decisions of a (Ti x Ti) level into row bit masks; texel
// k = r * Ti + c is handled by thread k.
template <int Ti>
__device__ __forceinline__ void store_rows(uint32_t* rows, int k, bool st) {
  const int lane = threadIdx.x & 31;
  const uint32_t b = __ballot_sync(0xffffffffu, st);
  if (k >= Ti * Ti) return;  // the whole row group lies past the level's last texel
  if (Ti >= 32) {
    if (lane == 0) rows[k / Ti] = b;
  } else if ((lane % Ti) == 0) {
    rows[k / Ti] = (b >> lane) & ((1u << (Ti & 31)) - 1u);
  }
}

// Level 0 with radius R: D_0 is the edge image itself.  Warp w owns tile rows
// [ROWS0 w, ROWS0 w + ROWS0), lane = column; the lane takes the horizontal sums of the
// ROWS0 + 2R rows it needs from their bit windows (a table of exact window sums where
// one is given) and the vertical taps from registers.
template <int R>
__device__ __forceinline__ void level0_blur(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  // rows per group: a group's horizontal sums (GR + 2R rows) stay in registers; one group
  // of 8 rows per warp at Table 1's level-0 radius 3 computes 14 row sums where two groups
  // of 4 computed 20 (the mask launch 34.1 -> 31.9 us at 3840x2160)
  constexpr int GR = R <= 3 ? 8 : 4;
  constexpr int NH = GR + 2 * R;
  constexpr uint32_t WMASK = (1u << (2 * R + 1)) - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool use_lut = m.lut0 != nullptr && (1 << (2 * R + 1)) <= MASK_LUT_MAX;
  const int b = EX - R + lane;           // first staged column of the lane's window
  const int k = b >> 5, sh = b & 31;
  float g[2 * R + 1];
#pragma unroll
  for (int t = 0; t <= 2 * R; ++t) g[t] = m.g[0][t];
  const int x = x0 + lane;
#pragma unroll 1
  for (int ty0 = ROWS0 * warp; ty0 < ROWS0 * (warp + 1); ty0 += GR) {
    float h[NH];
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < NH; ++j) {
      const uint4 row = sm.E[MG + ty0 - R + j];
      const uint32_t lo = k == 0 ? row.x : row.y, hi = k == 0 ? row.y : row.z;
      const uint32_t win = __funnelshift_r(lo, hi, sh) & WMASK;
      any |= win;
      h[j] = use_lut ? sm.lut[win] : window_sum(win, sm.g[0]);
    }
    const bool blur = __any_sync(0xffffffffu, any != 0u);
#pragma unroll
    for (int rr = 0; rr < GR; ++rr) {
      float s = 0.0f;
      if (blur) {
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t) s = fmaf(g[t], h[rr + t], s);
      }
      const int y = y0 + ty0 + rr;
      const bool inside = x < m.W && y < m.H;
      if (m.a0c) {
        sm.a0t[ty0 + rr][lane] = s;
      } else if (inside) {
        m.alpha[0][(size_t)y * m.W + x] = s;
        m.stencil[0][(size_t)y * m.W + x] = s > 0.0f ? 1 : 0;
      }
      const uint32_t bits = __ballot_sync(0xffffffffu, inside && s > 0.0f);
      if (lane == 0) sm.S[0][ty0 + rr] = bits;
    }
  }
}

// Level I >= 1 with blur radius R, nesting from level P (P < 0: none).
template <int I, int R, int P>
__device__ __forceinline__ void blur_level(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  constexpr int Ti = TS >> I, DN = Ti + 2 * R;
  constexpr uint32_t WMASK = (1u << (2 * R + 1)) - 1u;
  const int tid = threadIdx.x;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const int Wi = m.Wi[I], Hi = m.Hi[I];
  uint32_t d = 0;
  if (tid < DN) {
    d = d_row<I, R>(sm, tid);
    sm.D[tid] = d;
  }
  // no edge within reach of the tile: a_I = 0 here and both passes would add only zeros
  const bool blur = __syncthreads_or(d != 0u) != 0;
  if (blur) {
    const float* lut = m.lut[I];
    for (int k = tid; k < DN * Ti; k += MTHREADS) {
      const int r = k / Ti, c = k - r * Ti;
      const uint32_t win = (sm.D[r] >> c) & WMASK;
      sm.h[k] = lut ? __ldg(lut + win) : window_sum(win, sm.g[I]);
    }
  }
  __syncthreads();
  for (int base = 0; base < Ti * Ti; base += MTHREADS) {
    const int k = base + tid;
    const int r = k / Ti, c = k - r * Ti;
    const bool mine = k < Ti * Ti;
    float s = 0.0f;
    if (mine && blur) {
#pragma unroll
      for (int t = 0; t <= 2 * R; ++t) s = fmaf(m.g[I][t], sm.h[(r + t) * Ti + c], s);
    }
    bool st = s > 0.0f;
    if (P >= 0 && mine) {
      // inclusive nesting: any set child in the previous enabled finer level
      constexpr int F = P >= 0 ? I - P : 0, GP = 1 << F;
      uint32_t rows = 0;
#pragma unroll
      for (int j = 0; j < GP; ++j) rows |= sm.S[P >= 0 ? P : 0][r * GP + j];
      st = st || ((rows >> (c * GP)) & ((1u << GP) - 1u)) != 0u;
    }
    const int qx = q0x + c, qy = q0y + r;
    const bool inside = mine && qx < Wi && qy < Hi;
    st = st && inside;
    if (inside) {
      m.alpha[I][(size_t)qy * Wi + qx] = s;
      m.stencil[I][(size_t)qy * Wi + qx] = st ? 1 : 0;
    }
    store_rows<Ti>(sm.S[I], k, st);
  }
}

template <int I, int P>
__device__ __forceinline__ void blur_dispatch(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  if (I == 0) {
    switch (m.R[0]) {
      case 1: level0_blur<1>(m, sm, x0, y0); break;
      case 2: level0_blur<2>(m, sm, x0, y0); break;
      case 3: level0_blur<3>(m, sm, x0, y0); break;
      case 4: level0_blur<4>(m, sm, x0, y0); break;
      case 5: level0_blur<5>(m, sm, x0, y0); break;
      default: level0_blur<6>(m, sm, x0, y0); break;
    }
    return;
  }
  constexpr int J = I > 0 ? I : 1;
  switch (m.R[J]) {
    case 1: blur_level<J, 1, P>(m, sm, x0, y0); break;
    case 2: blur_level<J, 2, P>(m, sm, x0, y0); break;
    case 3: blur_level<J, 3, P>(m, sm, x0, y0); break;
    case 4: blur_level<J, 4, P>(m, sm, x0, y0); break;
    case 5: blur_level<J, 5, P>(m, sm, x0, y0); break;
    default: blur_level<J, 6, P>(m, sm, x0, y0); break;
  }
}

// Level I written as a constant (mode 1: a = 1, S = 1; mode 2: a = 0, S = 0).  Reads no
// shared memory, so it needs no barrier before it.
template <int I>
__device__ __forceinline__ void fill_level(const MaskParams& m, MaskSmem& sm, int x0, int y0, int mode) {
  constexpr int Ti = TS >> I;
  const int q0x = x0 >> I, q0y = y0 >> I;
  const float av = mode == 1 ? 1.0f : 0.0f;
  const uint8_t sv = mode == 1 ? 1 : 0;
  for (int base = 0; base < Ti * Ti; base += MTHREADS) {
    const int k = base + threadIdx.x;
    const int r = k / Ti, c = k - r * Ti;
    const bool inside = k < Ti * Ti && q0x + c < m.Wi[I] && q0y + r < m.Hi[I];
    if (I == 0 && m.a0c) {
      if (k < Ti * Ti) sm.a0t[r][c] = av;
    } else if (inside && m.alpha[I]) {
      m.alpha[I][(size_t)(q0y + r) * m.Wi[I] + q0x + c] = av;
      m.stencil[I][(size_t)(q0y + r) * m.Wi[I] + q0x + c] = sv;
    }
    store_rows<Ti>(sm.S[I], k, inside && mode == 1);
  }
}

// Level I, whose previous enabled finer level is P (-1: none).
template <int I, int P>
__device__ __forceinline__ void do_level(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  const int mode = m.mode[I];
  if (mode == 0) blur_dispatch<I, P>(m, sm, x0, y0);
  else fill_level<I>(m, sm, x0, y0, mode);
}

// The levels in order; blurred levels are 0..2 (the coarsest, at most 3, is a fill).
// Shared-memory order: level I's stencil rows are written before level I+1's first
// barrier and read after it; D and h of level I+1 are written after level I's last
// reads of them (its second barrier, and level I+1's first).
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

// Level patterns compiled on their own, so that the kernel holds only the code they run
// (the generic kernel carries every radius of every level, and its instruction footprint
// stalls warps on instruction fetch):
//   MASK_SIG_T1_4: four levels, levels 0-2 blurred with radii 3, 5, 6 (Table 1's SSAO and
//                  soft-shadow rows, sigma^2 = 0.924, 1.848, 3.696);
//   MASK_SIG_T1_GI: four levels, level 1 disabled, levels 0 and 2 blurred with radius 3
//                  (Table 1's SSGI rows);
//   MASK_SIG_T1_3: three levels, levels 0 and 1 blurred with radii 3 and 5.
// The steps and their order are those of all_levels for the same configuration.
enum { MASK_SIG_ANY = 0, MASK_SIG_T1_4 = 1, MASK_SIG_T1_GI = 2, MASK_SIG_T1_3 = 3 };

template <int SIG>
__device__ __forceinline__ void all_levels_sig(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  if constexpr (SIG == MASK_SIG_T1_4) {
    level0_blur<3>(m, sm, x0, y0);
    blur_level<1, 5, 0>(m, sm, x0, y0);
    blur_level<2, 6, 1>(m, sm, x0, y0);
    fill_level<3>(m, sm, x0, y0, m.mode[3]);
  } else if constexpr (SIG == MASK_SIG_T1_GI) {
    level0_blur<3>(m, sm, x0, y0);
    fill_level<1>(m, sm, x0, y0, 2);
    blur_level<2, 3, 0>(m, sm, x0, y0);
    fill_level<3>(m, sm, x0, y0, m.mode[3]);
  } else if constexpr (SIG == MASK_SIG_T1_3) {
    level0_blur<3>(m, sm, x0, y0);
    blur_level<1, 5, 0>(m, sm, x0, y0);
    fill_level<2>(m, sm, x0, y0, m.mode[2]);
  } else {
    all_levels(m, sm, x0, y0);
  }
}

// ---- frame mode: the work lists of every enabled level, written by the mask kernel
//
// Each tile reserves room for its set texels of each level with one atomicAdd on the
// level's count (zero before the launch), then writes them there in tile-local
// row-major order.  The order of the tiles within a list is whatever order the tiles
// reached their atomics; shading never depends on it (every entry is shaded and stored
// on its own), and the count is exact.
__device__ __forceinline__ void frame_lists(const MaskParams& m, MaskSmem& sm, int x0, int y0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (warp == 0) {
    uint32_t mine = 0;  // lane i: level i's count
#pragma unroll
    for (int i = 0; i < MRR_MAX_LEVELS; ++i) {
      const uint32_t pc = (i < m.L && lane < (TS >> i)) ? (uint32_t)__popc(sm.S[i][lane]) : 0u;
      uint32_t inc = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane < (TS >> i)) sm.rowpre[i][lane] = inc - pc;
      const uint32_t cnt = __shfl_sync(0xffffffffu, inc, 31);
      if (lane == i) mine = cnt;
    }
    // the levels' reservations go out together (one round trip, not four)
    uint32_t start = 0u;
    if (lane < m.L && m.mode[lane] != 2) {
      start = mine ? atomicAdd(m.counts + lane, mine) : 0u;
      sm.excl[lane] = start;
    }
  }
  __syncthreads();
  // level 0: warp w owns rows ROWS0 w .. ROWS0 w + ROWS0 - 1, lane = column
  if (m.mode[0] != 2) {
    const size_t cap = (size_t)m.Wi[0] * m.Hi[0];
#pragma unroll
    for (int rr = 0; rr < ROWS0; ++rr) {
      const int r = ROWS0 * warp + rr;
      const uint32_t bits = sm.S[0][r];
      if ((bits >> lane) & 1u) {
        const size_t pos = (size_t)sm.excl[0] + sm.rowpre[0][r] + __popc(bits & ((1u << lane) - 1u));
        if (pos < cap) {
          m.list[0][pos] = ((uint32_t)(y0 + r) << 16) | (uint32_t)(x0 + lane);
          m.a0c[pos] = sm.a0t[r][lane];
        }
      }
    }
  }
#pragma unroll
  for (int i = 1; i < MRR_MAX_LEVELS; ++i) {
    if (i >= m.L || m.mode[i] == 2) continue;
    const int Ti = TS >> i;
    for (int k = threadIdx.x; k < Ti * Ti; k += MTHREADS) {
      const int r = k / Ti, c = k - r * Ti;
      const uint32_t bits = sm.S[i][r];
      if ((bits >> c) & 1u) {
        const size_t pos = (size_t)sm.excl[i] + sm.rowpre[i][r] + __popc(bits & ((1u << c) - 1u));
        if (pos < (size_t)m.Wi[i] * m.Hi[i])
          m.list[i][pos] = ((uint32_t)((y0 >> i) + r) << 16) | (uint32_t)((x0 >> i) + c);
      }
    }
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
  if (m.ebits) {
    // bit-packed edge image: the three words of each staged row
    for (int k = threadIdx.x; k < ER * EWORDS; k += MTHREADS) {
      const int r = k / EWORDS, w = k - r * EWORDS;
      const int y = y0 - MG + r, wx = (x0 >> 5) - 1 + w;
      uint32_t v = 0u;
      if (y >= 0 && y < H && wx >= 0 && wx < m.ewords) v = __ldg(m.ebits + (size_t)y * m.ewords + wx);
      Ew[4 * r + w] = v;
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
  __syncthreads();
  all_levels_sig<SIG>(m, sm, x0, y0);
  if (m.a0c) frame_lists(m, sm, x0, y0);
  if (m.label) {
    __syncthreads();
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
