/*
 * scenegen.c -- seeded synthetic inputs for the multi-resolution rendering path.
 *
 * This module produces INPUTS only: a procedural scene (ground plane, axis-aligned
 * boxes, spheres), its G-buffer (linear view depth + view-space normals + direct-lit
 * colour) ray-cast through pixel centres, a light-space shadow map ray-cast from a
 * light camera, and the seeded sample tables (hemisphere kernel, unit-disk taps)
 * that the lighting effects draw.  It contains none of the method's arithmetic
 * (edges, masks, shading, blending); both the CPU oracle and the CUDA path consume
 * its outputs.  The paper evaluates on rasterised mesh scenes (Sec. 5); these
 * seeded scenes stand in for them.
 *
 * Everything is computed in double and rounded once to float.  No transcendental
 * function is used for the camera (tan 30 deg = 1/sqrt(3)); the sample tables use
 * cos/sin/sqrt in double, rounded once to float.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define SG_MAX_BOXES 256
#define SG_MAX_SPHERES 256

typedef struct { double lo[3], hi[3], alb[3]; } sg_box;
typedef struct { double c[3], r, alb[3]; } sg_sphere;
typedef struct {
  int nb, ns;
  sg_box b[SG_MAX_BOXES];
  sg_sphere s[SG_MAX_SPHERES];
  double ground_alb[3];
  double bmin[3], bmax[3]; /* bounds of all boxes and spheres */
} sg_scene;

/* SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then mix. */
static uint64_t sm64(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double u01(uint64_t *s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }
static double urange(uint64_t *s, double lo, double hi) { return lo + (hi - lo) * u01(s); }

/* Fixed draw order: per box sx, sy, sz in [0.2,1.5], cx, cz in [-3,3] (boxes rest on y=0);
 * per sphere r in [0.1,0.8], cx, cz in [-3,3] (centre y=r); then albedo rgb = 0.1+0.8u
 * for the ground, every box, every sphere. */
static void make_scene(uint64_t seed, int nb, int ns, sg_scene *sc) {
  uint64_t st = seed;
  if (nb > SG_MAX_BOXES) nb = SG_MAX_BOXES;
  if (ns > SG_MAX_SPHERES) ns = SG_MAX_SPHERES;
  if (nb < 0) nb = 0;
  if (ns < 0) ns = 0;
  sc->nb = nb;
  sc->ns = ns;
  for (int i = 0; i < nb; ++i) {
    double sx = urange(&st, 0.2, 1.5), sy = urange(&st, 0.2, 1.5), sz = urange(&st, 0.2, 1.5);
    double cx = urange(&st, -3.0, 3.0), cz = urange(&st, -3.0, 3.0);
    sg_box *b = &sc->b[i];
    b->lo[0] = cx - 0.5 * sx; b->hi[0] = cx + 0.5 * sx;
    b->lo[1] = 0.0;           b->hi[1] = sy;
    b->lo[2] = cz - 0.5 * sz; b->hi[2] = cz + 0.5 * sz;
  }
  for (int i = 0; i < ns; ++i) {
    double r = urange(&st, 0.1, 0.8);
    double cx = urange(&st, -3.0, 3.0), cz = urange(&st, -3.0, 3.0);
    sg_sphere *p = &sc->s[i];
    p->r = r; p->c[0] = cx; p->c[1] = r; p->c[2] = cz;
  }
  for (int k = 0; k < 3; ++k) sc->ground_alb[k] = urange(&st, 0.1, 0.9);
  for (int i = 0; i < nb; ++i) for (int k = 0; k < 3; ++k) sc->b[i].alb[k] = urange(&st, 0.1, 0.9);
  for (int i = 0; i < ns; ++i) for (int k = 0; k < 3; ++k) sc->s[i].alb[k] = urange(&st, 0.1, 0.9);
  for (int k = 0; k < 3; ++k) { sc->bmin[k] = 1e30; sc->bmax[k] = -1e30; }
  for (int i = 0; i < nb; ++i) for (int k = 0; k < 3; ++k) {
    if (sc->b[i].lo[k] < sc->bmin[k]) sc->bmin[k] = sc->b[i].lo[k];
    if (sc->b[i].hi[k] > sc->bmax[k]) sc->bmax[k] = sc->b[i].hi[k];
  }
  for (int i = 0; i < ns; ++i) for (int k = 0; k < 3; ++k) {
    if (sc->s[i].c[k] - sc->s[i].r < sc->bmin[k]) sc->bmin[k] = sc->s[i].c[k] - sc->s[i].r;
    if (sc->s[i].c[k] + sc->s[i].r > sc->bmax[k]) sc->bmax[k] = sc->s[i].c[k] + sc->s[i].r;
  }
}

/* Ray o + t*d against the whole scene; returns the nearest t in (tmin, inf) or -1.
 * On a hit, n gets the unit world normal and alb the albedo. */
static double trace(const sg_scene *sc, const double o[3], const double d[3], double tmin,
                    double n[3], double alb[3], int *id) {
  double best = -1.0;
  *id = -1;
  /* ground plane y = 0 */
  if (d[1] < 0.0 && o[1] > 0.0) {
    double t = -o[1] / d[1];
    if (t > tmin) {
      best = t;
      *id = 0;
      n[0] = 0.0; n[1] = 1.0; n[2] = 0.0;
      memcpy(alb, sc->ground_alb, sizeof(double) * 3);
    }
  }
  if (sc->nb + sc->ns == 0) return best;
  /* early out: slab test against the bounds of all objects */
  {
    double t0 = tmin, t1 = 1e300;
    for (int k = 0; k < 3; ++k) {
      if (d[k] == 0.0) {
        if (o[k] < sc->bmin[k] || o[k] > sc->bmax[k]) return best;
      } else {
        double a = (sc->bmin[k] - o[k]) / d[k], b = (sc->bmax[k] - o[k]) / d[k];
        if (a > b) { double tt = a; a = b; b = tt; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
      }
    }
    if (t0 > t1) return best;
  }
  for (int i = 0; i < sc->nb; ++i) {
    const sg_box *bx = &sc->b[i];
    double t0 = -1e300, t1 = 1e300;
    int ax = -1;
    int miss = 0;
    for (int k = 0; k < 3; ++k) {
      if (d[k] == 0.0) {
        if (o[k] < bx->lo[k] || o[k] > bx->hi[k]) { miss = 1; break; }
      } else {
        double a = (bx->lo[k] - o[k]) / d[k], b = (bx->hi[k] - o[k]) / d[k];
        if (a > b) { double tt = a; a = b; b = tt; }
        if (a > t0) { t0 = a; ax = k; }
        if (b < t1) t1 = b;
      }
    }
    if (miss || t0 > t1 || ax < 0) continue;
    if (t0 > tmin && (best < 0.0 || t0 < best)) {
      best = t0;
      *id = 1 + i;
      n[0] = n[1] = n[2] = 0.0;
      n[ax] = d[ax] > 0.0 ? -1.0 : 1.0;
      memcpy(alb, bx->alb, sizeof(double) * 3);
    }
  }
  for (int i = 0; i < sc->ns; ++i) {
    const sg_sphere *sp = &sc->s[i];
    double oc[3] = {o[0] - sp->c[0], o[1] - sp->c[1], o[2] - sp->c[2]};
    double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - sp->r * sp->r;
    double disc = b * b - a * c;
    if (disc < 0.0) continue;
    double t = (-b - sqrt(disc)) / a;
    if (t > tmin && (best < 0.0 || t < best)) {
      best = t;
      *id = 1 + sc->nb + i;
      for (int k = 0; k < 3; ++k) n[k] = (o[k] + t * d[k] - sp->c[k]) / sp->r;
      double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int k = 0; k < 3; ++k) n[k] /= len;
      memcpy(alb, sp->alb, sizeof(double) * 3);
    }
  }
  return best;
}

static void normalize3(double v[3]) {
  double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= l; v[1] /= l; v[2] /= l;
}
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Look-at basis: forward f = normalize(target - eye), right r = normalize(f x up),
 * up u = r x f.  View space is (right, up, -forward), camera looks down -z. */
static void look_at(const double eye[3], const double tgt[3], double r[3], double u[3], double f[3]) {
  const double up[3] = {0.0, 1.0, 0.0};
  for (int k = 0; k < 3; ++k) f[k] = tgt[k] - eye[k];
  normalize3(f);
  cross3(f, up, r);
  normalize3(r);
  cross3(r, f, u);
}

/* Camera description handed to consumers as floats (rounded once from double):
 * cam[0..2] eye, [3..5] right, [6..8] up, [9..11] forward, [12] tan(fov/2),
 * [13] near, [14] far. */
void sg_camera(const double eye[3], const double tgt[3], double tan_half, double nearp, double farp,
               float cam[15]) {
  double r[3], u[3], f[3];
  look_at(eye, tgt, r, u, f);
  for (int k = 0; k < 3; ++k) {
    cam[k] = (float)eye[k];
    cam[3 + k] = (float)r[k];
    cam[6 + k] = (float)u[k];
    cam[9 + k] = (float)f[k];
  }
  cam[12] = (float)tan_half;
  cam[13] = (float)nearp;
  cam[14] = (float)farp;
}

/* G-buffer of scene(seed) seen from eye -> target with a vertical half-angle whose
 * tangent is tan_half, for a W x H image (row 0 = top).  Rays pass through pixel
 * centres (x+1/2, y+1/2).  depth = linear view depth (distance along the forward
 * axis); a miss or a hit at depth >= far is sky: depth = far, normal = 0.
 * normal4 = view-space unit normal (xyz, w = 0).  color4 = albedo * max(0, n.l)
 * for the directional light l = normalize(1,2,1) with unit irradiance (w = 0).
 * objid = 0 for the ground, 1+i for box i, 1+nb+i for sphere i, -1 for sky.
 * Any output pointer may be NULL. */
void sg_gbuffer(uint64_t seed, int nb, int ns, int W, int H, const double eye[3], const double tgt[3],
                double tan_half, double nearp, double farp, float *depth, float *normal4, float *color4,
                int32_t *objid) {
  static sg_scene sc_static; /* large: keep it off the stack */
  sg_scene *sc = &sc_static;
  make_scene(seed, nb, ns, sc);
  double r[3], u[3], f[3];
  look_at(eye, tgt, r, u, f);
  double aspect = (double)W / (double)H;
  double l[3] = {1.0, 2.0, 1.0};
  normalize3(l);
#pragma omp parallel for schedule(dynamic, 4)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      double sx = (2.0 * (x + 0.5) / W - 1.0) * tan_half * aspect;
      double sy = (1.0 - 2.0 * (y + 0.5) / H) * tan_half;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = f[k] + sx * r[k] + sy * u[k];
      double n[3] = {0, 0, 0}, alb[3] = {0, 0, 0};
      int hit_id;
      double t = trace(sc, eye, d, nearp, n, alb, &hit_id);
      size_t i = (size_t)y * W + x;
      int sky = !(t > 0.0) || t >= farp;
      if (depth) depth[i] = (float)(sky ? farp : t);
      if (normal4) {
        if (sky) {
          normal4[4 * i] = normal4[4 * i + 1] = normal4[4 * i + 2] = normal4[4 * i + 3] = 0.0f;
        } else {
          double vx = n[0] * r[0] + n[1] * r[1] + n[2] * r[2];
          double vy = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
          double vz = -(n[0] * f[0] + n[1] * f[1] + n[2] * f[2]);
          normal4[4 * i] = (float)vx;
          normal4[4 * i + 1] = (float)vy;
          normal4[4 * i + 2] = (float)vz;
          normal4[4 * i + 3] = 0.0f;
        }
      }
      if (color4) {
        double nl = n[0] * l[0] + n[1] * l[1] + n[2] * l[2];
        if (nl < 0.0 || sky) nl = 0.0;
        for (int k = 0; k < 3; ++k) color4[4 * i + k] = (float)(alb[k] * nl);
        color4[4 * i + 3] = 0.0f;
      }
      if (objid) objid[i] = sky ? -1 : hit_id;
    }
  }
}

/* World-space hit position of the ray through pixel (x,y) (for tests of the view
 * reconstruction): returns 1 on a hit (xyz written), 0 for sky. */
int sg_pixel_world(uint64_t seed, int nb, int ns, int W, int H, const double eye[3], const double tgt[3],
                   double tan_half, double nearp, double farp, int x, int y, double out[3]) {
  static sg_scene sc_static;
  sg_scene *sc = &sc_static;
  make_scene(seed, nb, ns, sc);
  double r[3], u[3], f[3];
  look_at(eye, tgt, r, u, f);
  double aspect = (double)W / (double)H;
  double sx = (2.0 * (x + 0.5) / W - 1.0) * tan_half * aspect;
  double sy = (1.0 - 2.0 * (y + 0.5) / H) * tan_half;
  double d[3], n[3], alb[3];
  int hit_id;
  for (int k = 0; k < 3; ++k) d[k] = f[k] + sx * r[k] + sy * u[k];
  double t = trace(sc, eye, d, nearp, n, alb, &hit_id);
  if (!(t > 0.0) || t >= farp) return 0;
  for (int k = 0; k < 3; ++k) out[k] = eye[k] + t * d[k];
  return 1;
}

/* Shadow map: linear light depth (distance along the light's forward axis) of
 * scene(seed) seen from the light camera, S x S texels through texel centres,
 * square frustum with half-angle tangent tan_half; a miss or depth >= far is far. */
void sg_shadow_map(uint64_t seed, int nb, int ns, int S, const double eye[3], const double tgt[3],
                   double tan_half, double nearp, double farp, float *sm) {
  static sg_scene sc_static;
  sg_scene *sc = &sc_static;
  make_scene(seed, nb, ns, sc);
  double r[3], u[3], f[3];
  look_at(eye, tgt, r, u, f);
#pragma omp parallel for schedule(dynamic, 4)
  for (int y = 0; y < S; ++y) {
    for (int x = 0; x < S; ++x) {
      double sx = (2.0 * (x + 0.5) / S - 1.0) * tan_half;
      double sy = (1.0 - 2.0 * (y + 0.5) / S) * tan_half;
      double d[3], n[3], alb[3];
      int hit_id;
      for (int k = 0; k < 3; ++k) d[k] = f[k] + sx * r[k] + sy * u[k];
      double t = trace(sc, eye, d, nearp, n, alb, &hit_id);
      sm[(size_t)y * S + x] = (float)((!(t > 0.0) || t >= farp) ? farp : t);
    }
  }
}

/* Seeded cosine-weighted hemisphere kernel (tangent frame, +z = normal):
 * direction (sqrt(u1) cos(2 pi u2), sqrt(u1) sin(2 pi u2), sqrt(1-u1)) scaled by
 * 0.1 + 0.9 (j/N)^2 so that samples cluster near the centre; out = N x 4 floats. */
void sg_hemisphere_kernel(uint64_t seed, int N, float *out4) {
  uint64_t st = seed;
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < N; ++j) {
    double u1 = u01(&st), u2 = u01(&st);
    double rr = sqrt(u1), ph = two_pi * u2;
    double s = (double)j / (double)N;
    double len = 0.1 + 0.9 * s * s;
    out4[4 * j] = (float)(rr * cos(ph) * len);
    out4[4 * j + 1] = (float)(rr * sin(ph) * len);
    out4[4 * j + 2] = (float)(sqrt(1.0 - u1) * len);
    out4[4 * j + 3] = 0.0f;
  }
}

/* Seeded uniform points in the unit disk: (sqrt(u1) cos(2 pi u2), sqrt(u1) sin(2 pi u2)). */
void sg_disk_taps(uint64_t seed, int N, float *out2) {
  uint64_t st = seed;
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < N; ++j) {
    double u1 = u01(&st), u2 = u01(&st);
    double rr = sqrt(u1), ph = two_pi * u2;
    out2[2 * j] = (float)(rr * cos(ph));
    out2[2 * j + 1] = (float)(rr * sin(ph));
  }
}

/* Poisson arrival gaps and uniform picks for the serving mix: gaps[i] = -ln(1-u)/rate,
 * pick[i] = floor(u' * n_choices). */
void sg_poisson_stream(uint64_t seed, int n, double rate, int n_choices, double *gaps, int32_t *pick) {
  uint64_t st = seed;
  for (int i = 0; i < n; ++i) {
    double u = u01(&st);
    gaps[i] = -log(1.0 - u) / rate;
    int k = (int)(u01(&st) * n_choices);
    if (k >= n_choices) k = n_choices - 1;
    pick[i] = k;
  }
}
