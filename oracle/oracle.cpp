// oracle.cpp -- plain, slow CPU oracle for the multi-resolution rendering method of
// Besenthal, Maisch and Ropinski, "Multi-Resolution Rendering for Computationally
// Expensive Lighting Effects" (arXiv 1906.04576).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg may load this library; the product path never does.  It shares no
// code, header, table or constant generator with the CUDA library: the two meet only
// in the seeded inputs (scene G-buffer, camera floats, sample tables) that both take.
//
// Every function follows the paper's steps in order, with no blocking or fusion:
//   Sec. 3.1  edge image from depth (2nd derivative) and normal (1st derivative)
//             discontinuities, plus shadow discontinuities for soft shadows;
//             downsample to each level, Gaussian blur with variance sigma_i^2
//             (Table 1), inclusive nesting of the levels (Sec. 3.1, Fig. 2/3);
//   Sec. 4.1  stencil = [mask > 0]; each sub-image shaded only where its stencil is set;
//             optionally a bilateral blur of the rendered sub-images;
//   Sec. 2.4  the effects (SSAO, PCSS soft shadows, SSGI) -- the paper gives no
//             formulas, so the readings below are fixed in the design notes;
//   Sec. 4.2  bilinear upsampling of every sub-image to full size and the sequential
//             blend of Eq. (1), from the coarsest level to the finest; optionally the
//             step-wise chain of Sec. 3.3 instead;
//   Sec. 6    optionally sample-count levels: levels above 0 rendered at full
//             resolution with fewer samples, blended without upsampling.
// T = float is the parity oracle (discrete decisions in the kernels' precision, FP32);
// T = double is the FP64 reference for error statements.  The build uses
// -ffp-contract=off: a multiply-add is fused only where the source writes std::fma
// (one rounding), every other operation is rounded on its own, in source order.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Parameters of one render, as plain floats/ints (mirrored by a ctypes Structure).
struct orc_params {
  int effect;            // 0 = SSAO, 1 = soft shadow mapping (PCSS), 2 = SSGI
  int width, height;     // full-resolution W x H
  int num_levels;        // L <= 4: level i has scale 2^-i (the paper's sub-image i+1)
  float sigma2[4];       // Table 1 blur variances, in level-i texels
  float weight[4];       // Table 1 blend weights w_i
  int enabled[4];        // 0 disables a level (SSGI skips the 1/2 level, Sec. 4)
  float depth_rel;       // depth edge: |second difference| > depth_rel * depth
  float normal_cos;      // normal edge: dot of neighbouring normals < normal_cos
  int force_level0;      // every pixel assigned to level 0 (a_0 = 1, S_0 = 1)
  int samples;           // N, SSAO / SSGI hemisphere samples
  float radius;          // r, world-space sampling radius
  float ao_bias;         // SSAO depth bias
  float gi_min_dist2;    // SSGI distance clamp (squared)
  const float* kernel;   // N x 4 hemisphere kernel (tangent frame)
  int blocker_samples;   // PCSS blocker-search taps
  int pcf_samples;       // PCSS filter taps
  const float* blocker_taps;  // unit disk, 2 floats each
  const float* pcf_taps;      // unit disk, 2 floats each
  float light_size;      // world-space side of the square area light
  float shadow_bias;     // light-depth bias
  int store_half;        // level buffers rounded to binary16 (FP16 storage)
  float cam[15];         // eye, right, up, forward, tan(fov/2), near, far
  float light[15];       // the light camera, same layout
  int shadow_size;       // S, shadow map is S x S
  int blur[4];           // 1: level i's sub-image gets the bilateral blur of Sec. 4.1
  float blur_depth_rel;  // that blur's depth test: |d' - d| <= blur_depth_rel * d
  int merge_mode;        // 0: direct upsampling (Sec. 4.2); 1: step-wise chain (Sec. 3.3);
                         // 2: direct upsampling with depth-aware (bilateral) taps (Sec. 3.3)
  int sample_levels;     // 1: levels above 0 at full resolution with fewer samples (Sec. 6)
  int pyramid_gathers;   // 1: SSAO on levels above 0 gathers depth from the level's point samples
  int gather_level;      // set per call by shade_level: the level whose samples the gathers read
  int disjoint;          // 1: complementary tiles without overlap (the variant Sec. 3.1 rejects)
};

}  // extern "C"

namespace {

template <typename T> struct V3 { T x, y, z; };

// Pinhole camera constants, derived in double from the float inputs, rounded once to T.
// slope_x(x) = (x + 1/2) * ax - bx,  slope_y(y) = by - (y + 1/2) * ay, and the
// inverse map X = (slope_x + bx) * kx,  Y = (by - slope_y) * ky (pixel coordinates
// whose integer part is the pixel index).
template <typename T> struct View {
  int W, H;
  T ax, bx, kx, ay, by, ky, nearp, farp;
};

template <typename T> View<T> make_view(int W, int H, float tan_half, float nearp, float farp) {
  double th = tan_half;
  double tx = th * ((double)W / (double)H);
  View<T> v;
  v.W = W;
  v.H = H;
  v.ax = (T)(2.0 * tx / (double)W);
  v.bx = (T)tx;
  v.kx = (T)((double)W / (2.0 * tx));
  v.ay = (T)(2.0 * th / (double)H);
  v.by = (T)th;
  v.ky = (T)((double)H / (2.0 * th));
  v.nearp = (T)nearp;
  v.farp = (T)farp;
  return v;
}

// Level geometry.  Level i has W_i = ceil(W / 2^i) texels per row; texel q covers the
// full-resolution block [2^i q, 2^i (q+1)) and is a point sample of the pixel
// s_i(q) = min(2^i q + o_i, W - 1), with o_0 = 0 and o_i = 2^(i-1) (the block centre).
inline int level_dim(int n, int i) { return (n + (1 << i) - 1) >> i; }
inline int level_origin(int i) { return i == 0 ? 0 : (1 << (i - 1)); }
inline int level_sample(int q, int i, int n) { return std::min((q << i) + level_origin(i), n - 1); }

// Round a float to the nearest binary16 value (ties to even), returned as a float.
// Written from the IEEE 754 binary16 format: 10 fraction bits, exponent range
// [-14, 15], subnormal quantum 2^-24, overflow to infinity above 65504 after rounding.
float round_to_half(float f) {
  if (std::isnan(f)) return f;
  double a = std::fabs((double)f);
  if (a == 0.0) return f;
  int e;
  std::frexp(a, &e);                 // a = m * 2^e with m in [0.5, 1): exponent of a is e-1
  int exp_a = e - 1;
  if (exp_a < -14) exp_a = -14;      // subnormal range: fixed quantum 2^-24
  double q = std::ldexp(1.0, exp_a - 10);
  double r = std::nearbyint(a / q) * q;  // default rounding mode: to nearest, ties to even
  if (r > 65504.0) r = INFINITY;
  return (float)(f < 0 ? -r : r);
}

// ---------------------------------------------------------------- effects (Sec. 2.4)

// Orthonormal basis around a unit normal n (Duff et al. 2017), sign chosen by n.z >= 0.
template <typename T> void make_basis(const V3<T>& n, V3<T>& t, V3<T>& b) {
  T s = n.z >= T(0) ? T(1) : T(-1);
  T a = T(-1) / (s + n.z);
  T c = n.x * n.y * a;
  t.x = T(1) + s * n.x * n.x * a;
  t.y = s * c;
  t.z = -s * n.x;
  b.x = c;
  b.y = s + n.y * n.y * a;
  b.z = -n.y;
}

struct Inputs {
  const float* depth;   // [H][W]
  const float* normal;  // [H][W][4]
  const float* color;   // [H][W][4] or null
  const float* smap;    // [S][S] or null
};

// View-space position of pixel (x, y) at linear depth d: the pixel centre's ray slopes
// sx = (x + 1/2) ax - bx and sy = by - (y + 1/2) ay (each one fused multiply-add), times d.
template <typename T> V3<T> view_pos(const View<T>& v, int x, int y, T d) {
  T sx = std::fma((T)x + T(0.5), v.ax, -v.bx);
  T sy = std::fma(-((T)y + T(0.5)), v.ay, v.by);
  V3<T> p = {sx * d, sy * d, -d};
  return p;
}

// Sample point S = P + k.x (r T) + k.y (r B) + k.z (r N), accumulated with fused
// multiply-adds in the order k.x, k.y, k.z.
template <typename T>
V3<T> sample_point(const V3<T>& P, const V3<T>& tr, const V3<T>& br, const V3<T>& nr, T kx, T ky, T kz) {
  V3<T> S;
  S.x = std::fma(kz, nr.x, std::fma(ky, br.x, std::fma(kx, tr.x, P.x)));
  S.y = std::fma(kz, nr.y, std::fma(ky, br.y, std::fma(kx, tr.y, P.y)));
  S.z = std::fma(kz, nr.z, std::fma(ky, br.z, std::fma(kx, tr.z, P.z)));
  return S;
}

// Projection of a view-space point with depth dS = -S.z >= near to pixel coordinates:
// inv = 1 / dS (correctly rounded), X = (S.x inv + bx) kx, Y = (by - S.y inv) ky, the
// bracketed terms as fused multiply-adds.  The pixel index is the integer part.
template <typename T> void project(const View<T>& v, const V3<T>& S, T dS, T& X, T& Y) {
  T inv = T(1) / dS;
  X = std::fma(S.x, inv, v.bx) * v.kx;
  Y = std::fma(-S.y, inv, v.by) * v.ky;
}

template <typename T> V3<T> scale3(const V3<T>& a, T s) {
  V3<T> r = {s * a.x, s * a.y, s * a.z};
  return r;
}

template <typename T> V3<T> load_normal(const Inputs& in, int W, int x, int y) {
  const float* n = in.normal + 4 * ((size_t)y * W + x);
  V3<T> r = {(T)n[0], (T)n[1], (T)n[2]};
  return r;
}

// SSAO (Mittring 2007; Bavoil et al. 2008), our reading: N samples S = P + k_x (rT) +
// k_y (rB) + k_z (rN) in the normal's hemisphere; each is projected to its pixel, and it is
// occluded when the depth buffer there lies in front of it by more than the bias and
// within the radius of the shaded point.  AO = 1 - occluded / N; sky is 1.
// Pyramid gathers (p.gather_level = i > 0): the depth buffer is read at level i's point
// samples instead -- the sample pixel s_i(Q) of the level-i block Q the projected pixel
// lies in, i.e. a depth pyramid made by point sampling.
template <typename T> T ssao_at(const orc_params& p, const View<T>& v, const Inputs& in, int x, int y) {
  const int W = v.W, H = v.H;
  T d = (T)in.depth[(size_t)y * W + x];
  if (d >= v.farp) return T(1);
  V3<T> n = load_normal<T>(in, W, x, y);
  V3<T> P = view_pos(v, x, y, d);
  V3<T> t, b;
  make_basis(n, t, b);
  const T r = (T)p.radius, bias = (T)p.ao_bias;
  const V3<T> tr = scale3(t, r), br = scale3(b, r), nr = scale3(n, r);
  int occ = 0;
  for (int j = 0; j < p.samples; ++j) {
    T kx = (T)p.kernel[4 * j], ky = (T)p.kernel[4 * j + 1], kz = (T)p.kernel[4 * j + 2];
    V3<T> S = sample_point(P, tr, br, nr, kx, ky, kz);
    T dS = -S.z;
    if (dS < v.nearp) continue;
    T X, Y;
    project(v, S, dS, X, Y);
    if (!(X >= T(0) && X < (T)W)) continue;
    if (!(Y >= T(0) && Y < (T)H)) continue;
    int ix = (int)X, iy = (int)Y;
    if (p.gather_level > 0) {  // pyramid gathers: the depth of the pixel's level-i block
      ix = level_sample(ix >> p.gather_level, p.gather_level, W);
      iy = level_sample(iy >> p.gather_level, p.gather_level, H);
    }
    T ds = (T)in.depth[(size_t)iy * W + ix];
    if (ds >= v.farp) continue;
    if (ds <= dS - bias && std::fabs(d - ds) < r) occ += 1;
  }
  return T(1) - (T)occ / (T)p.samples;
}

// SSGI (Ritschel et al. 2009), our reading: the same hemisphere samples (radius r); each
// projected pixel s contributes its direct light C_s with the form factor
// max(0, n.w) max(0, -n_s.w) / max(|D|^2, dmin^2), D = P_s - P, w = D/|D|, for
// 0 < |D|^2 <= r^2.  GI = (r^2 / N) * sum; sky is 0.
template <typename T>
void ssgi_at(const orc_params& p, const View<T>& v, const Inputs& in, int x, int y, T out[3]) {
  const int W = v.W, H = v.H;
  out[0] = out[1] = out[2] = T(0);
  T d = (T)in.depth[(size_t)y * W + x];
  if (d >= v.farp) return;
  V3<T> n = load_normal<T>(in, W, x, y);
  V3<T> P = view_pos(v, x, y, d);
  V3<T> t, b;
  make_basis(n, t, b);
  const T r = (T)p.radius;
  const T r2 = r * r;
  const T dmin2 = (T)p.gi_min_dist2;
  const V3<T> tr = scale3(t, r), br = scale3(b, r), nr = scale3(n, r);
  T acc[3] = {T(0), T(0), T(0)};
  for (int j = 0; j < p.samples; ++j) {
    T kx = (T)p.kernel[4 * j], ky = (T)p.kernel[4 * j + 1], kz = (T)p.kernel[4 * j + 2];
    V3<T> S = sample_point(P, tr, br, nr, kx, ky, kz);
    T dS = -S.z;
    if (dS < v.nearp) continue;
    T X, Y;
    project(v, S, dS, X, Y);
    if (!(X >= T(0) && X < (T)W)) continue;
    if (!(Y >= T(0) && Y < (T)H)) continue;
    int ix = (int)X, iy = (int)Y;
    T ds = (T)in.depth[(size_t)iy * W + ix];
    if (ds >= v.farp) continue;
    V3<T> Ps = view_pos(v, ix, iy, ds);
    V3<T> D = {Ps.x - P.x, Ps.y - P.y, Ps.z - P.z};
    T dd = std::fma(D.z, D.z, std::fma(D.y, D.y, D.x * D.x));
    if (dd > r2 || dd == T(0)) continue;
    T il = T(1) / std::sqrt(dd);
    V3<T> w = {D.x * il, D.y * il, D.z * il};
    V3<T> ns = load_normal<T>(in, W, ix, iy);
    T c1 = std::fma(n.z, w.z, std::fma(n.y, w.y, n.x * w.x));
    T c2 = -std::fma(ns.z, w.z, std::fma(ns.y, w.y, ns.x * w.x));
    T g = std::max(T(0), c1) * std::max(T(0), c2) / std::max(dd, dmin2);
    const float* C = in.color + 4 * ((size_t)iy * W + ix);
    acc[0] = std::fma((T)C[0], g, acc[0]);
    acc[1] = std::fma((T)C[1], g, acc[1]);
    acc[2] = std::fma((T)C[2], g, acc[2]);
  }
  T scale = r2 / (T)p.samples;
  out[0] = acc[0] * scale;
  out[1] = acc[1] * scale;
  out[2] = acc[2] * scale;
}

// Light-space coordinates of a visible pixel: receiver depth zr and shadow-map texel
// coordinates (Xt, Yt).  Returns false when the point is not in front of the light's
// near plane.  World position = eye + P.x right + P.y up + d forward.
template <typename T> struct LightView {
  T e[3], r[3], u[3], f[3];
  T tl, kl, nearp, farp;
  int S;
};

template <typename T> LightView<T> make_light(const orc_params& p) {
  LightView<T> L;
  for (int k = 0; k < 3; ++k) {
    L.e[k] = (T)p.light[k];
    L.r[k] = (T)p.light[3 + k];
    L.u[k] = (T)p.light[6 + k];
    L.f[k] = (T)p.light[9 + k];
  }
  L.tl = (T)p.light[12];
  L.nearp = (T)p.light[13];
  L.farp = (T)p.light[14];
  L.S = p.shadow_size;
  L.kl = (T)((double)p.shadow_size / (2.0 * (double)p.light[12]));
  return L;
}

template <typename T>
bool light_coords(const orc_params& p, const View<T>& v, const LightView<T>& L, int x, int y, T d, T& zr,
                  T& Xt, T& Yt) {
  V3<T> P = view_pos(v, x, y, d);
  T wp[3], lv[3];
  for (int k = 0; k < 3; ++k) {
    T e = (T)p.cam[k], r = (T)p.cam[3 + k], u = (T)p.cam[6 + k], f = (T)p.cam[9 + k];
    wp[k] = e + (P.x * r + P.y * u + d * f);
  }
  for (int k = 0; k < 3; ++k) lv[k] = wp[k] - L.e[k];
  zr = lv[0] * L.f[0] + lv[1] * L.f[1] + lv[2] * L.f[2];
  T lx = lv[0] * L.r[0] + lv[1] * L.r[1] + lv[2] * L.r[2];
  T ly = lv[0] * L.u[0] + lv[1] * L.u[1] + lv[2] * L.u[2];
  if (!(zr > L.nearp)) return false;
  T inv = T(1) / zr;
  Xt = (lx * inv + L.tl) * L.kl;
  Yt = (L.tl - ly * inv) * L.kl;
  return true;
}

// One-sample hard shadow (Sec. 3.1: "one sample per pixel"): 1 lit, 0 shadowed.
template <typename T>
int hard_shadow_at(const orc_params& p, const View<T>& v, const LightView<T>& L, const Inputs& in, int x,
                   int y) {
  T d = (T)in.depth[(size_t)y * v.W + x];
  T zr, Xt, Yt;
  if (!light_coords(p, v, L, x, y, d, zr, Xt, Yt)) return 1;
  const T S = (T)L.S;
  if (!(Xt >= T(0) && Xt < S && Yt >= T(0) && Yt < S)) return 1;
  T z = (T)in.smap[(size_t)(int)Yt * L.S + (int)Xt];
  return z >= zr - (T)p.shadow_bias ? 1 : 0;
}

// Soft shadow mapping: shadow map (Williams 1978) + percentage-closer filtering
// (Reeves et al. 1987) with the PCSS penumbra estimate (Fernando 2005), our reading:
// blocker search over a disk of radius (l/2)(zr - n)/(zr n) (tangent units) scaled to
// texels, average blocker depth zb, filter radius (l/2)(zr - zb)/(zb zr), then the lit
// fraction of the PCF taps.  Off-map taps are lit; sky is 1.
template <typename T>
T ssm_at(const orc_params& p, const View<T>& v, const LightView<T>& L, const Inputs& in, int x, int y) {
  T d = (T)in.depth[(size_t)y * v.W + x];
  if (d >= v.farp) return T(1);
  T zr, Xt, Yt;
  if (!light_coords(p, v, L, x, y, d, zr, Xt, Yt)) return T(1);
  const T S = (T)L.S;
  const T bias = (T)p.shadow_bias;
  const T hl = (T)p.light_size * T(0.5);
  T rs = hl * (zr - L.nearp) / (zr * L.nearp) * L.kl;
  T sum = T(0);
  int cnt = 0;
  for (int j = 0; j < p.blocker_samples; ++j) {
    T tx = std::fma((T)p.blocker_taps[2 * j], rs, Xt);
    T ty = std::fma((T)p.blocker_taps[2 * j + 1], rs, Yt);
    if (!(tx >= T(0) && tx < S && ty >= T(0) && ty < S)) continue;
    T zb = (T)in.smap[(size_t)(int)ty * L.S + (int)tx];
    if (zb < zr - bias) {
      sum = sum + zb;
      cnt += 1;
    }
  }
  if (cnt == 0) return T(1);
  T zavg = sum / (T)cnt;
  T rf = hl * (zr - zavg) / (zavg * zr) * L.kl;
  int lit = 0;
  for (int j = 0; j < p.pcf_samples; ++j) {
    T tx = std::fma((T)p.pcf_taps[2 * j], rf, Xt);
    T ty = std::fma((T)p.pcf_taps[2 * j + 1], rf, Yt);
    if (!(tx >= T(0) && tx < S && ty >= T(0) && ty < S)) {
      lit += 1;
      continue;
    }
    T z = (T)in.smap[(size_t)(int)ty * L.S + (int)tx];
    if (z >= zr - bias) lit += 1;
  }
  return (T)lit / (T)p.pcf_samples;
}

int channels(const orc_params& p) { return p.effect == 2 ? 3 : 1; }

// Effect value at full-resolution pixel (x, y), C channels.
template <typename T>
void shade_at(const orc_params& p, const View<T>& v, const LightView<T>& L, const Inputs& in, int x, int y,
              T* out) {
  if (p.effect == 0) {
    out[0] = ssao_at(p, v, in, x, y);
  } else if (p.effect == 1) {
    out[0] = ssm_at(p, v, L, in, x, y);
  } else {
    ssgi_at(p, v, in, x, y, out);
  }
}

template <typename T> bool is_sky(const View<T>& v, const Inputs& in, int x, int y) {
  return (T)in.depth[(size_t)y * v.W + x] >= v.farp;
}

// ---------------------------------------------------------------- Sec. 3.1 edges

// Edge image E: a non-sky pixel is an edge when
//   (a) any in-image 4-neighbour is sky;
//   (b) the second difference of depth along x or y exceeds depth_rel times its depth
//       (an axis counts only when both neighbours are inside the image);
//   (c) the dot product with any in-image non-sky 4-neighbour's normal is below
//       normal_cos (first derivative of the normals);
//   (d) soft shadows only: its one-sample hard shadow differs from any in-image
//       non-sky 4-neighbour's (Sec. 3.1), combined with (a)-(c) by OR (maximum).
// Sky pixels are never edges.
template <typename T> void edges(const orc_params& p, const Inputs& in, uint8_t* E) {
  const int W = p.width, H = p.height;
  View<T> v = make_view<T>(W, H, p.cam[12], p.cam[13], p.cam[14]);
  std::vector<int> hs;
  if (p.effect == 1) {
    LightView<T> L = make_light<T>(p);
    hs.assign((size_t)W * H, 1);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        if (!is_sky(v, in, x, y)) hs[(size_t)y * W + x] = hard_shadow_at(p, v, L, in, x, y);
  }
  const T rel = (T)p.depth_rel, ncos = (T)p.normal_cos;
  const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      size_t i = (size_t)y * W + x;
      T d = (T)in.depth[i];
      if (d >= v.farp) {
        E[i] = 0;
        continue;
      }
      bool e = false;
      for (int k = 0; k < 4; ++k) {
        int nx = x + dx[k], ny = y + dy[k];
        if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
        if (is_sky(v, in, nx, ny)) e = true;
      }
      if (x > 0 && x < W - 1) {
        T lap = ((T)in.depth[i - 1] + (T)in.depth[i + 1]) - T(2) * d;
        if (std::fabs(lap) > rel * d) e = true;
      }
      if (y > 0 && y < H - 1) {
        T lap = ((T)in.depth[i - W] + (T)in.depth[i + W]) - T(2) * d;
        if (std::fabs(lap) > rel * d) e = true;
      }
      V3<T> n = load_normal<T>(in, W, x, y);
      for (int k = 0; k < 4; ++k) {
        int nx = x + dx[k], ny = y + dy[k];
        if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
        if (is_sky(v, in, nx, ny)) continue;
        V3<T> m = load_normal<T>(in, W, nx, ny);
        T dot = n.x * m.x + n.y * m.y + n.z * m.z;
        if (dot < ncos) e = true;
        if (p.effect == 1 && hs[(size_t)ny * W + nx] != hs[i]) e = true;
      }
      E[i] = e ? 1 : 0;
    }
  }
}

// ---------------------------------------------------------------- Sec. 3.1 masks

// Truncated, normalised Gaussian of variance sigma2: radius R = ceil(3 sigma),
// g_k = exp(-k^2 / (2 sigma2)) / sum_j exp(-j^2 / (2 sigma2)), k = -R..R, in double,
// rounded once to T.
template <typename T> int gauss_weights(double sigma2, T* g) {
  int R = (int)std::ceil(3.0 * std::sqrt(sigma2));
  std::vector<double> e(2 * R + 1);
  double sum = 0.0;
  for (int k = -R; k <= R; ++k) {
    e[k + R] = std::exp(-(double)(k * k) / (2.0 * sigma2));
    sum += e[k + R];
  }
  for (int k = 0; k <= 2 * R; ++k) g[k] = (T)(e[k] / sum);
  return R;
}

// Masks of all levels (Sec. 3.1, Table 1, Sec. 4.1):
//   D_i(q) = max of E over the block of q (the downsampled edge image);
//   a_i = horizontal then vertical truncated Gaussian of D_i with variance sigma_i^2,
//         taps in ascending order (one fused multiply-add per tap), zero outside the level;
//   S_i = [a_i > 0] (the stencil of Sec. 4.1);
//   nesting (Fig. 2/3): S_j(Q) |= S_k(q) for every q of the previous enabled finer
//         level k inside Q's block, so finer areas are included in coarser ones;
//   the coarsest level has a = 1 and S = 1 everywhere; disabled levels a = 0, S = 0;
//   force_level0: a_0 = 1 and S_0 = 1 everywhere.
// label(p) = the finest enabled level i whose stencil is set at p's block (p >> i).
template <typename T>
void masks(const orc_params& p, const uint8_t* E, T* const* a, uint8_t* const* S, uint8_t* label) {
  const int W = p.width, H = p.height, L = p.num_levels;
  int prev = -1;
  for (int i = 0; i < L; ++i) {
    const int Wi = level_dim(W, i), Hi = level_dim(H, i);
    const size_t ni = (size_t)Wi * Hi;
    if (!p.enabled[i]) {
      for (size_t k = 0; k < ni; ++k) {
        a[i][k] = T(0);
        S[i][k] = 0;
      }
      continue;
    }
    if (i == L - 1 || (i == 0 && p.force_level0)) {
      for (size_t k = 0; k < ni; ++k) {
        a[i][k] = T(1);
        S[i][k] = 1;
      }
    } else {
      std::vector<uint8_t> D(ni, 0);
      const int bs = 1 << i;
      for (int qy = 0; qy < Hi; ++qy)
        for (int qx = 0; qx < Wi; ++qx) {
          uint8_t m = 0;
          for (int y = qy * bs; y < std::min(qy * bs + bs, H); ++y)
            for (int x = qx * bs; x < std::min(qx * bs + bs, W); ++x) m = std::max(m, E[(size_t)y * W + x]);
          D[(size_t)qy * Wi + qx] = m;
        }
      T g[64];
      const int R = gauss_weights<T>((double)p.sigma2[i], g);
      std::vector<T> h(ni);
      for (int y = 0; y < Hi; ++y)
        for (int x = 0; x < Wi; ++x) {
          T s = T(0);
          for (int k = -R; k <= R; ++k) {
            int xx = x + k;
            if (xx < 0 || xx >= Wi) continue;
            s = std::fma(g[k + R], (T)D[(size_t)y * Wi + xx], s);
          }
          h[(size_t)y * Wi + x] = s;
        }
      for (int y = 0; y < Hi; ++y)
        for (int x = 0; x < Wi; ++x) {
          T s = T(0);
          for (int k = -R; k <= R; ++k) {
            int yy = y + k;
            if (yy < 0 || yy >= Hi) continue;
            s = std::fma(g[k + R], h[(size_t)yy * Wi + x], s);
          }
          a[i][(size_t)y * Wi + x] = s;
          S[i][(size_t)y * Wi + x] = s > T(0) ? 1 : 0;
        }
    }
    if (p.disjoint) {
      // Complementary tiles (Sec. 3.1, the variant without overlap): level i keeps only
      // the blocks of its own mask that no finer level has rendered any part of, so no
      // area is rendered twice.  Pixels of a block that a finer level rendered only in
      // part belong to no sub-image: the dead pixels of Fig. 4 (left).
      for (int qy = 0; qy < Hi; ++qy)
        for (int qx = 0; qx < Wi; ++qx) {
          if (!S[i][(size_t)qy * Wi + qx]) continue;
          bool covered = false;
          for (int f = 0; f < i && !covered; ++f) {
            if (!p.enabled[f]) continue;
            const int Wf = level_dim(W, f), Hf = level_dim(H, f), k = i - f;
            for (int y = qy << k; y < std::min((qy + 1) << k, Hf) && !covered; ++y)
              for (int x = qx << k; x < std::min((qx + 1) << k, Wf); ++x)
                if (S[f][(size_t)y * Wf + x]) {
                  covered = true;
                  break;
                }
          }
          if (covered) S[i][(size_t)qy * Wi + qx] = 0;
        }
    } else if (prev >= 0) {
      const int Wp = level_dim(W, prev), Hp = level_dim(H, prev);
      const int f = 1 << (i - prev);
      for (int qy = 0; qy < Hi; ++qy)
        for (int qx = 0; qx < Wi; ++qx) {
          uint8_t any = 0;
          for (int y = qy * f; y < std::min(qy * f + f, Hp); ++y)
            for (int x = qx * f; x < std::min(qx * f + f, Wp); ++x) any |= S[prev][(size_t)y * Wp + x];
          if (any) S[i][(size_t)qy * Wi + qx] = 1;
        }
    }
    prev = i;
  }
  if (label) {
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int lab = -1;
        for (int i = 0; i < L && lab < 0; ++i) {
          if (!p.enabled[i]) continue;
          const int Wi = level_dim(W, i);
          if (S[i][(size_t)(y >> i) * Wi + (x >> i)]) lab = i;
        }
        label[(size_t)y * W + x] = (uint8_t)lab;
      }
  }
}

// ---------------------------------------------------------------- Sec. 3.2 / 4.1

// Work list of level i: the texels with S_i = 1 in row-major order, packed (y << 16) | x.
int compact(int Wi, int Hi, const uint8_t* S, uint32_t* list) {
  int n = 0;
  for (int y = 0; y < Hi; ++y)
    for (int x = 0; x < Wi; ++x)
      if (S[(size_t)y * Wi + x]) list[n++] = ((uint32_t)y << 16) | (uint32_t)x;
  return n;
}

// Sub-image i: c_i(q) = effect at the full-resolution pixel s_i(q), for every q in the
// work list; texels outside it are left untouched.  C channels per texel.
template <typename T>
void shade_level(const orc_params& p0, const Inputs& in, int level, const uint32_t* list, int n, T* c) {
  orc_params p = p0;
  p.gather_level = (p0.pyramid_gathers && p0.effect == 0) ? level : 0;
  const int W = p.width, H = p.height, C = channels(p);
  const int Wi = level_dim(W, level);
  View<T> v = make_view<T>(W, H, p.cam[12], p.cam[13], p.cam[14]);
  LightView<T> L = make_light<T>(p);
#pragma omp parallel for schedule(dynamic, 256)
  for (int k = 0; k < n; ++k) {
    int qx = (int)(list[k] & 0xFFFFu), qy = (int)(list[k] >> 16);
    int x = level_sample(qx, level, W), y = level_sample(qy, level, H);
    T val[3];
    shade_at(p, v, L, in, x, y, val);
    for (int ch = 0; ch < C; ++ch) {
      T out = val[ch];
      if (p.store_half) out = (T)round_to_half((float)out);
      c[((size_t)qy * Wi + qx) * C + ch] = out;
    }
  }
}

// ---------------------------------------------------------------- Sec. 4.1 sub-image blur

// Bilateral blur of sub-image i (Sec. 4.1: the SSAO sub-images, above all the coarse
// ones, are blurred against sampling variance, and the blur must not take values from
// texels that were never rendered).  For every rendered texel q (S_i(q) = 1):
//   b_i(q) = sum_t w_t c_i(q + t) / sum_t w_t,
// the sums taken over the offsets t = (tx, ty) of the 5 x 5 window, tx, ty in -2..2, whose
// texel q + t is inside the level, rendered, and on q's surface:
//   |d(s_i(q + t)) - d(s_i(q))| <= blur_depth_rel * d(s_i(q)),
// d being the full-resolution depth at a texel's sample pixel s_i.  The spatial weight is
// w_t = B[tx] B[ty] with the binomial row B = (1, 4, 6, 4, 1) (Pascal's triangle, the
// discrete Gaussian of variance 1).  Both sums run over the window in row-major order;
// q itself always takes part, so the denominator is at least 36.  Texels outside the
// stencil are copied unchanged.
template <typename T>
void blur_level(const orc_params& p, const float* depth, int level, const uint8_t* S, const T* c, T* b) {
  const int W = p.width, H = p.height, C = channels(p);
  const int Wi = level_dim(W, level), Hi = level_dim(H, level);
  const T B[5] = {T(1), T(4), T(6), T(4), T(1)};
  const T rel = (T)p.blur_depth_rel;
#pragma omp parallel for schedule(static)
  for (int qy = 0; qy < Hi; ++qy) {
    for (int qx = 0; qx < Wi; ++qx) {
      const size_t q = (size_t)qy * Wi + qx;
      if (!S[q]) {
        for (int ch = 0; ch < C; ++ch) b[q * C + ch] = c[q * C + ch];
        continue;
      }
      const T d = (T)depth[(size_t)level_sample(qy, level, H) * W + level_sample(qx, level, W)];
      T num[3] = {T(0), T(0), T(0)}, den = T(0);
      for (int ty = -2; ty <= 2; ++ty) {
        for (int tx = -2; tx <= 2; ++tx) {
          const int ux = qx + tx, uy = qy + ty;
          if (ux < 0 || ux >= Wi || uy < 0 || uy >= Hi) continue;
          const size_t u = (size_t)uy * Wi + ux;
          if (!S[u]) continue;
          const T du = (T)depth[(size_t)level_sample(uy, level, H) * W + level_sample(ux, level, W)];
          if (!(std::fabs(du - d) <= rel * d)) continue;
          const T w = B[ty + 2] * B[tx + 2];
          for (int ch = 0; ch < C; ++ch) num[ch] = num[ch] + w * c[u * C + ch];
          den = den + w;
        }
      }
      for (int ch = 0; ch < C; ++ch) {
        T out = num[ch] / den;
        if (p.store_half) out = (T)round_to_half((float)out);
        b[q * C + ch] = out;
      }
    }
  }
}

// Sample-count levels (Sec. 6 proposes them for effects that must not be sub-sampled:
// a sub-image rendered at full resolution with fewer samples instead of at a lower
// resolution).  Level i >= 1 keeps its mask and work list, but every full-resolution
// pixel of each listed texel's block [2^i q, 2^i q + 2^i) (inside the image) is shaded;
// p carries the level's sample tables (the caller thins them).  c is [H][W] x C; pixels
// outside the listed blocks are left untouched.
template <typename T>
void shade_blocks(const orc_params& p, const Inputs& in, int level, const uint32_t* list, int n, T* c) {
  const int W = p.width, H = p.height, C = channels(p), B = 1 << level;
  View<T> v = make_view<T>(W, H, p.cam[12], p.cam[13], p.cam[14]);
  LightView<T> L = make_light<T>(p);
#pragma omp parallel for schedule(dynamic, 64)
  for (int k = 0; k < n; ++k) {
    const int qx = (int)(list[k] & 0xFFFFu), qy = (int)(list[k] >> 16);
    for (int dy = 0; dy < B; ++dy) {
      for (int dx = 0; dx < B; ++dx) {
        const int x = qx * B + dx, y = qy * B + dy;
        if (x >= W || y >= H) continue;
        T val[3];
        shade_at(p, v, L, in, x, y, val);
        for (int ch = 0; ch < C; ++ch) {
          T out = val[ch];
          if (p.store_half) out = (T)round_to_half((float)out);
          c[((size_t)y * W + x) * C + ch] = out;
        }
      }
    }
  }
}

// Naive full-resolution rendering (the comparison of Sec. 5): the effect at every pixel.
template <typename T> void shade_full(const orc_params& p, const Inputs& in, T* out) {
  const int W = p.width, H = p.height, C = channels(p);
  View<T> v = make_view<T>(W, H, p.cam[12], p.cam[13], p.cam[14]);
  LightView<T> L = make_light<T>(p);
#pragma omp parallel for schedule(dynamic, 1)
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      T val[3];
      shade_at(p, v, L, in, x, y, val);
      for (int ch = 0; ch < C; ++ch) out[((size_t)y * W + x) * C + ch] = val[ch];
    }
}

// ---------------------------------------------------------------- Sec. 4.2 blending

// Upsampling and Eq. (1).  Level texel q sits at full-resolution position 2^i q + o_i,
// so pixel p reads level coordinate u = (p - o_i) / 2^i; the four bilinear taps
// floor(u), floor(u)+1 are clamped to the level.  a_i is interpolated plainly; c_i is
// interpolated only over taps whose stencil is set, with the weights renormalised
// (unrendered texels hold no information, Sec. 3.3).  Starting from c' = the coarsest
// sub-image, every finer enabled level i is blended in:
//     alpha = min(w_i * a_i, 1),   c' = c_i * alpha + c' * (1 - alpha)
// (Eq. (1), read with c' on the right-hand side being the previous, coarser composite).
template <typename T>
void merge(const orc_params& p, T* const* a, uint8_t* const* S, T* const* c, T* out) {
  const int W = p.width, H = p.height, L = p.num_levels, C = channels(p);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      T cp[3] = {T(0), T(0), T(0)};
      bool first = true;
      for (int i = L - 1; i >= 0; --i) {
        if (!p.enabled[i]) continue;
        const int Wi = level_dim(W, i), Hi = level_dim(H, i);
        const T scale = (T)(1 << i);
        T ux = (T)(x - level_origin(i)) / scale;
        T uy = (T)(y - level_origin(i)) / scale;
        int x0 = (int)std::floor(ux), y0 = (int)std::floor(uy);
        T fx = ux - (T)x0, fy = uy - (T)y0;
        int xs[2] = {std::min(std::max(x0, 0), Wi - 1), std::min(std::max(x0 + 1, 0), Wi - 1)};
        int ys[2] = {std::min(std::max(y0, 0), Hi - 1), std::min(std::max(y0 + 1, 0), Hi - 1)};
        T w[4] = {(T(1) - fx) * (T(1) - fy), fx * (T(1) - fy), (T(1) - fx) * fy, fx * fy};
        size_t idx[4] = {(size_t)ys[0] * Wi + xs[0], (size_t)ys[0] * Wi + xs[1], (size_t)ys[1] * Wi + xs[0],
                         (size_t)ys[1] * Wi + xs[1]};
        T ahat = T(0);
        for (int k = 0; k < 4; ++k) ahat = ahat + w[k] * a[i][idx[k]];
        T alpha = std::min((T)p.weight[i] * ahat, T(1));
        if (!first && !(alpha > T(0))) continue;
        T num[3] = {T(0), T(0), T(0)}, den = T(0);
        for (int k = 0; k < 4; ++k) {
          if (!S[i][idx[k]]) continue;
          for (int ch = 0; ch < C; ++ch) num[ch] = num[ch] + w[k] * c[i][idx[k] * C + ch];
          den = den + w[k];
        }
        if (first) {
          for (int ch = 0; ch < C; ++ch) cp[ch] = num[ch] / den;
          first = false;
          continue;
        }
        for (int ch = 0; ch < C; ++ch) {
          T chat = num[ch] / den;
          cp[ch] = chat * alpha + cp[ch] * (T(1) - alpha);
        }
      }
      for (int ch = 0; ch < C; ++ch) out[((size_t)y * W + x) * C + ch] = cp[ch];
    }
  }
}

// Recomposition of complementary tiles (Sec. 3.1, the variant without overlap): pixel p
// takes the sub-image of the finest enabled level whose stencil covers it, interpolated
// bilinearly at p over that level's rendered taps only (weights renormalised), with no
// blending.  A pixel that no level covers, or whose covering level has no rendered tap of
// positive weight at p, is undefined: NaN (a dead pixel).
template <typename T>
void merge_disjoint(const orc_params& p, uint8_t* const* S, T* const* c, T* out) {
  const int W = p.width, H = p.height, L = p.num_levels, C = channels(p);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      T v[3] = {T(NAN), T(NAN), T(NAN)};
      for (int i = 0; i < L; ++i) {
        if (!p.enabled[i]) continue;
        const int Wi = level_dim(W, i), Hi = level_dim(H, i);
        if (!S[i][(size_t)(y >> i) * Wi + (x >> i)]) continue;
        const T scale = (T)(1 << i);
        T ux = (T)(x - level_origin(i)) / scale;
        T uy = (T)(y - level_origin(i)) / scale;
        int x0 = (int)std::floor(ux), y0 = (int)std::floor(uy);
        T fx = ux - (T)x0, fy = uy - (T)y0;
        int xs[2] = {std::min(std::max(x0, 0), Wi - 1), std::min(std::max(x0 + 1, 0), Wi - 1)};
        int ys[2] = {std::min(std::max(y0, 0), Hi - 1), std::min(std::max(y0 + 1, 0), Hi - 1)};
        T w[4] = {(T(1) - fx) * (T(1) - fy), fx * (T(1) - fy), (T(1) - fx) * fy, fx * fy};
        size_t idx[4] = {(size_t)ys[0] * Wi + xs[0], (size_t)ys[0] * Wi + xs[1], (size_t)ys[1] * Wi + xs[0],
                         (size_t)ys[1] * Wi + xs[1]};
        T num[3] = {T(0), T(0), T(0)}, den = T(0);
        for (int k = 0; k < 4; ++k) {
          if (!S[i][idx[k]] || !(w[k] > T(0))) continue;
          for (int ch = 0; ch < C; ++ch) num[ch] = num[ch] + w[k] * c[i][idx[k] * C + ch];
          den = den + w[k];
        }
        if (den > T(0))
          for (int ch = 0; ch < C; ++ch) v[ch] = num[ch] / den;
        break;
      }
      for (int ch = 0; ch < C; ++ch) out[((size_t)y * W + x) * C + ch] = v[ch];
    }
  }
}

// Direct upsampling with bilateral taps (Sec. 3.3 cites Tomasi and Manduchi's bilateral
// filter for upsampling without mixing in unrelated pixels).  As merge above, except that
// c_i is interpolated over the rendered taps that also lie on the pixel's surface:
// tap k (texel Q_k) takes weight w_k when S_i(Q_k) = 1 and
//   |d(s_i(Q_k)) - d(p)| <= blur_depth_rel * d(p),
// d the full-resolution depth (the blur's depth test); when no tap passes, the rendered
// taps are used as in merge.  a_i stays plain bilinear.  depth is [H][W].
template <typename T>
void merge_bilateral(const orc_params& p, const float* depth, T* const* a, uint8_t* const* S, T* const* c,
                     T* out) {
  const int W = p.width, H = p.height, L = p.num_levels, C = channels(p);
  const T rel = (T)p.blur_depth_rel;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      const T dp = (T)depth[(size_t)y * W + x];
      T cp[3] = {T(0), T(0), T(0)};
      bool first = true;
      for (int i = L - 1; i >= 0; --i) {
        if (!p.enabled[i]) continue;
        const int Wi = level_dim(W, i), Hi = level_dim(H, i);
        const T scale = (T)(1 << i);
        T ux = (T)(x - level_origin(i)) / scale;
        T uy = (T)(y - level_origin(i)) / scale;
        int x0 = (int)std::floor(ux), y0 = (int)std::floor(uy);
        T fx = ux - (T)x0, fy = uy - (T)y0;
        int xs[2] = {std::min(std::max(x0, 0), Wi - 1), std::min(std::max(x0 + 1, 0), Wi - 1)};
        int ys[2] = {std::min(std::max(y0, 0), Hi - 1), std::min(std::max(y0 + 1, 0), Hi - 1)};
        T w[4] = {(T(1) - fx) * (T(1) - fy), fx * (T(1) - fy), (T(1) - fx) * fy, fx * fy};
        int tx[4] = {xs[0], xs[1], xs[0], xs[1]}, ty[4] = {ys[0], ys[0], ys[1], ys[1]};
        T ahat = T(0);
        for (int k = 0; k < 4; ++k) ahat = ahat + w[k] * a[i][(size_t)ty[k] * Wi + tx[k]];
        T alpha = std::min((T)p.weight[i] * ahat, T(1));
        if (!first && !(alpha > T(0))) continue;
        T num[3] = {T(0), T(0), T(0)}, den = T(0);
        T numb[3] = {T(0), T(0), T(0)}, denb = T(0);
        for (int k = 0; k < 4; ++k) {
          const size_t q = (size_t)ty[k] * Wi + tx[k];
          if (!S[i][q]) continue;
          for (int ch = 0; ch < C; ++ch) num[ch] = num[ch] + w[k] * c[i][q * C + ch];
          den = den + w[k];
          const T dq = (T)depth[(size_t)level_sample(ty[k], i, H) * W + level_sample(tx[k], i, W)];
          if (!(std::fabs(dq - dp) <= rel * dp)) continue;
          for (int ch = 0; ch < C; ++ch) numb[ch] = numb[ch] + w[k] * c[i][q * C + ch];
          denb = denb + w[k];
        }
        if (denb > T(0)) {
          for (int ch = 0; ch < C; ++ch) num[ch] = numb[ch];
          den = denb;
        }
        if (first) {
          for (int ch = 0; ch < C; ++ch) cp[ch] = num[ch] / den;
          first = false;
          continue;
        }
        for (int ch = 0; ch < C; ++ch) {
          T chat = num[ch] / den;
          cp[ch] = chat * alpha + cp[ch] * (T(1) - alpha);
        }
      }
      for (int ch = 0; ch < C; ++ch) out[((size_t)y * W + x) * C + ch] = cp[ch];
    }
  }
}

// Step-wise blending (Sec. 3.3), the alternative to the direct upsampling above: the
// sub-images are merged from the coarsest upwards, each finer enabled level i blended,
// at its own resolution, with the composite of the levels below it scaled up to level
// i's grid; the full-resolution image is the composite at level 0.  Starting from
// comp = c_{L-1} (the coarsest level is rendered everywhere), for every finer level i
// (descending; disabled levels above 0 are skipped, so a step may span several
// octaves) and every texel q of level i:
//   u = (2^i q + o_i - o_j) / 2^j   (q's position in texels of the previous level j)
//   up = bilinear interpolation of comp at u (taps floor(u), floor(u) + 1 clamped; comp
//        is defined everywhere, so no renormalisation)
//   comp_i(q) = c_i(q) * alpha + up * (1 - alpha),  alpha = min(w_i a_i(q), 1),
//               where S_i(q) = 1 and alpha > 0;  comp_i(q) = up elsewhere.
// Level 0 takes part as any other level when enabled, and is the last step either way.
template <typename T>
void merge_stepwise(const orc_params& p, T* const* a, uint8_t* const* S, T* const* c, T* out) {
  const int W = p.width, H = p.height, L = p.num_levels, C = channels(p);
  int j = L - 1;
  std::vector<T> comp(c[j], c[j] + (size_t)level_dim(W, j) * level_dim(H, j) * C);
  for (int i = L - 2; i >= 0; --i) {
    if (i > 0 && !p.enabled[i]) continue;
    const int Wi = level_dim(W, i), Hi = level_dim(H, i), Wj = level_dim(W, j), Hj = level_dim(H, j);
    const T scale = (T)(1 << j);
    std::vector<T> next((size_t)Wi * Hi * C);
#pragma omp parallel for schedule(static)
    for (int qy = 0; qy < Hi; ++qy) {
      for (int qx = 0; qx < Wi; ++qx) {
        T ux = (T)((qx << i) + level_origin(i) - level_origin(j)) / scale;
        T uy = (T)((qy << i) + level_origin(i) - level_origin(j)) / scale;
        int x0 = (int)std::floor(ux), y0 = (int)std::floor(uy);
        T fx = ux - (T)x0, fy = uy - (T)y0;
        int xs[2] = {std::min(std::max(x0, 0), Wj - 1), std::min(std::max(x0 + 1, 0), Wj - 1)};
        int ys[2] = {std::min(std::max(y0, 0), Hj - 1), std::min(std::max(y0 + 1, 0), Hj - 1)};
        T w[4] = {(T(1) - fx) * (T(1) - fy), fx * (T(1) - fy), (T(1) - fx) * fy, fx * fy};
        size_t idx[4] = {(size_t)ys[0] * Wj + xs[0], (size_t)ys[0] * Wj + xs[1], (size_t)ys[1] * Wj + xs[0],
                         (size_t)ys[1] * Wj + xs[1]};
        const size_t q = (size_t)qy * Wi + qx;
        T up[3] = {T(0), T(0), T(0)};
        for (int k = 0; k < 4; ++k)
          for (int ch = 0; ch < C; ++ch) up[ch] = up[ch] + w[k] * comp[idx[k] * C + ch];
        T alpha = T(0);
        if (p.enabled[i] && S[i][q]) alpha = std::min((T)p.weight[i] * a[i][q], T(1));
        for (int ch = 0; ch < C; ++ch)
          next[q * C + ch] = alpha > T(0) ? c[i][q * C + ch] * alpha + up[ch] * (T(1) - alpha) : up[ch];
      }
    }
    comp.swap(next);
    j = i;
  }
  std::copy(comp.begin(), comp.end(), out);
}

// Blending of sample-count levels: every sub-image is full resolution, so nothing is
// upsampled but the masks.  Per pixel p, from c' = c_{L-1}(p) (the coarsest level is
// rendered everywhere) over every finer enabled level i: if p's texel at level i,
// (p_x >> i, p_y >> i), is rendered, alpha = min(w_i a_i(p), 1) with a_i(p) interpolated
// bilinearly exactly as in the direct merge above, and c' = c_i(p) alpha + c' (1 - alpha)
// where alpha > 0; a pixel whose texel is not rendered keeps c' (its value does not exist).
template <typename T>
void merge_samples(const orc_params& p, T* const* a, uint8_t* const* S, T* const* c, T* out) {
  const int W = p.width, H = p.height, L = p.num_levels, C = channels(p);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      const size_t pix = (size_t)y * W + x;
      T cp[3] = {T(0), T(0), T(0)};
      for (int ch = 0; ch < C; ++ch) cp[ch] = c[L - 1][pix * C + ch];
      for (int i = L - 2; i >= 0; --i) {
        if (!p.enabled[i]) continue;
        const int Wi = level_dim(W, i), Hi = level_dim(H, i);
        if (!S[i][(size_t)(y >> i) * Wi + (x >> i)]) continue;
        const T scale = (T)(1 << i);
        T ux = (T)(x - level_origin(i)) / scale;
        T uy = (T)(y - level_origin(i)) / scale;
        int x0 = (int)std::floor(ux), y0 = (int)std::floor(uy);
        T fx = ux - (T)x0, fy = uy - (T)y0;
        int xs[2] = {std::min(std::max(x0, 0), Wi - 1), std::min(std::max(x0 + 1, 0), Wi - 1)};
        int ys[2] = {std::min(std::max(y0, 0), Hi - 1), std::min(std::max(y0 + 1, 0), Hi - 1)};
        T w[4] = {(T(1) - fx) * (T(1) - fy), fx * (T(1) - fy), (T(1) - fx) * fy, fx * fy};
        size_t idx[4] = {(size_t)ys[0] * Wi + xs[0], (size_t)ys[0] * Wi + xs[1], (size_t)ys[1] * Wi + xs[0],
                         (size_t)ys[1] * Wi + xs[1]};
        T ahat = T(0);
        for (int k = 0; k < 4; ++k) ahat = ahat + w[k] * a[i][idx[k]];
        T alpha = std::min((T)p.weight[i] * ahat, T(1));
        if (!(alpha > T(0))) continue;
        for (int ch = 0; ch < C; ++ch) cp[ch] = c[i][pix * C + ch] * alpha + cp[ch] * (T(1) - alpha);
      }
      for (int ch = 0; ch < C; ++ch) out[pix * C + ch] = cp[ch];
    }
  }
}

Inputs make_inputs(const float* depth, const float* normal, const float* color, const float* smap) {
  Inputs in;
  in.depth = depth;
  in.normal = normal;
  in.color = color;
  in.smap = smap;
  return in;
}

}  // namespace

// ---------------------------------------------------------------- C entry points
extern "C" {

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_level_dim(int n, int level) { return level_dim(n, level); }
int orc_level_sample(int q, int level, int n) { return level_sample(q, level, n); }
float orc_round_to_half(float f) { return round_to_half(f); }

int orc_gauss_weights_f32(double sigma2, float* g) { return gauss_weights<float>(sigma2, g); }
int orc_gauss_weights_f64(double sigma2, double* g) { return gauss_weights<double>(sigma2, g); }

#define ORC_STAGES(SUF, T)                                                                                  \
  void orc_edges_##SUF(const orc_params* p, const float* depth, const float* normal, const float* smap,     \
                       uint8_t* E) {                                                                         \
    edges<T>(*p, make_inputs(depth, normal, nullptr, smap), E);                                              \
  }                                                                                                          \
  void orc_hard_shadow_##SUF(const orc_params* p, const float* depth, const float* smap, int32_t* out) {    \
    View<T> v = make_view<T>(p->width, p->height, p->cam[12], p->cam[13], p->cam[14]);                      \
    LightView<T> L = make_light<T>(*p);                                                                      \
    Inputs in = make_inputs(depth, nullptr, nullptr, smap);                                                  \
    for (int y = 0; y < p->height; ++y)                                                                      \
      for (int x = 0; x < p->width; ++x)                                                                     \
        out[(size_t)y * p->width + x] = is_sky(v, in, x, y) ? -1 : hard_shadow_at(*p, v, L, in, x, y);     \
  }                                                                                                          \
  void orc_masks_##SUF(const orc_params* p, const uint8_t* E, T* const* a, uint8_t* const* S,               \
                       uint8_t* label) {                                                                     \
    masks<T>(*p, E, a, S, label);                                                                            \
  }                                                                                                          \
  void orc_shade_level_##SUF(const orc_params* p, const float* depth, const float* normal,                  \
                             const float* color, const float* smap, int level, const uint32_t* list, int n, \
                             T* c) {                                                                         \
    shade_level<T>(*p, make_inputs(depth, normal, color, smap), level, list, n, c);                         \
  }                                                                                                          \
  void orc_shade_full_##SUF(const orc_params* p, const float* depth, const float* normal,                   \
                            const float* color, const float* smap, T* out) {                                \
    shade_full<T>(*p, make_inputs(depth, normal, color, smap), out);                                         \
  }                                                                                                          \
  void orc_shade_pixel_##SUF(const orc_params* p, const float* depth, const float* normal,                  \
                             const float* color, const float* smap, int x, int y, T* out) {                 \
    View<T> v = make_view<T>(p->width, p->height, p->cam[12], p->cam[13], p->cam[14]);                      \
    LightView<T> L = make_light<T>(*p);                                                                      \
    shade_at(*p, v, L, make_inputs(depth, normal, color, smap), x, y, out);                                  \
  }                                                                                                          \
  void orc_make_basis_##SUF(const double* n, T* out) {                                                     \
    V3<T> nn = {(T)n[0], (T)n[1], (T)n[2]}, t, b;                                                            \
    make_basis(nn, t, b);                                                                                    \
    T v[9] = {t.x, t.y, t.z, b.x, b.y, b.z, nn.x, nn.y, nn.z};                                               \
    for (int k = 0; k < 9; ++k) out[k] = v[k];                                                               \
  }                                                                                                          \
  void orc_view_pos_##SUF(const orc_params* p, int x, int y, double d, T* out) {                            \
    View<T> v = make_view<T>(p->width, p->height, p->cam[12], p->cam[13], p->cam[14]);                      \
    V3<T> P = view_pos(v, x, y, (T)d);                                                                       \
    out[0] = P.x;                                                                                            \
    out[1] = P.y;                                                                                            \
    out[2] = P.z;                                                                                            \
  }                                                                                                          \
  void orc_merge_##SUF(const orc_params* p, T* const* a, uint8_t* const* S, T* const* c, T* out) {          \
    merge<T>(*p, a, S, c, out);                                                                              \
  }                                                                                                          \
  void orc_merge_bilateral_##SUF(const orc_params* p, const float* depth, T* const* a, uint8_t* const* S,   \
                                 T* const* c, T* out) {                                                       \
    merge_bilateral<T>(*p, depth, a, S, c, out);                                                             \
  }                                                                                                          \
  void orc_shade_blocks_##SUF(const orc_params* p, const float* depth, const float* normal,                  \
                              const float* color, const float* smap, int level, const uint32_t* list, int n,\
                              T* c) {                                                                        \
    shade_blocks<T>(*p, make_inputs(depth, normal, color, smap), level, list, n, c);                        \
  }                                                                                                          \
  void orc_merge_disjoint_##SUF(const orc_params* p, uint8_t* const* S, T* const* c, T* out) {               \
    merge_disjoint<T>(*p, S, c, out);                                                                        \
  }                                                                                                          \
  void orc_merge_samples_##SUF(const orc_params* p, T* const* a, uint8_t* const* S, T* const* c, T* out) {  \
    merge_samples<T>(*p, a, S, c, out);                                                                      \
  }                                                                                                          \
  void orc_merge_stepwise_##SUF(const orc_params* p, T* const* a, uint8_t* const* S, T* const* c, T* out) { \
    merge_stepwise<T>(*p, a, S, c, out);                                                                     \
  }                                                                                                          \
  void orc_blur_level_##SUF(const orc_params* p, const float* depth, int level, const uint8_t* S,           \
                            const T* c, T* b) {                                                              \
    blur_level<T>(*p, depth, level, S, c, b);                                                                \
  }

ORC_STAGES(f32, float)
ORC_STAGES(f64, double)

int orc_compact(int Wi, int Hi, const uint8_t* S, uint32_t* list) { return compact(Wi, Hi, S, list); }

}  // extern "C"
