"""Pins of the oracle's geometry against facts that do not come from the oracle itself.

* The tangent frame the effects build around a normal (Duff et al. 2017, the basis the
  SSAO and SSGI readings of Sec. 2.4 use) must be orthonormal and right-handed for every
  unit normal, including those facing away from the view axis, and give the natural
  frame at the pole.
* SSAO on a constant depth buffer with a tilted normal: which samples are occluded follows
  from the sample's displacement along the view axis alone, a closed form of the frame.
* SSGI's magnitude: one sample whose projected pixel holds a chosen surface gives the
  value of the form factor computed here from the pinhole camera, above and below the
  distance clamp, with the r^2 / N scale.
* Soft shadows' edge term (Sec. 3.1, "one sample per pixel"): a half-plane occluder over
  the ground adds edges exactly where a pixel's hard shadow, computed here from the camera
  and light definitions, differs from a 4-neighbour's.
"""
import math

import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from conftest import flat_normals, synthetic_frame

TAN30 = math.tan(math.radians(30.0))


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def _normals():
    rng = np.random.default_rng(7)
    v = rng.standard_normal((400, 3))
    out = [_unit(x) for x in v]
    # the pole, the antipode, the equator and their neighbourhoods
    for z in (1.0, -1.0, 1 - 1e-7, -1 + 1e-7, -1 + 1e-3, 1e-9, -1e-9, 0.0):
        out.append(_unit([math.sqrt(max(0.0, 1 - z * z)) * 0.6, math.sqrt(max(0.0, 1 - z * z)) * 0.8, z]))
    for ax in np.eye(3):
        out += [ax, -ax]
    return out


# ----------------------------------------------------------------- tangent frame

@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_basis_is_orthonormal_and_right_handed(precision, tol):
    for n in _normals():
        F = orc.make_basis(n, precision).astype(np.float64)
        t, b, nn = F
        assert np.allclose(nn, n, atol=tol)
        # rows of a rotation: unit length, pairwise orthogonal, t x b = n
        assert np.allclose(F @ F.T, np.eye(3), atol=4 * tol), (n, F)
        assert np.allclose(np.cross(t, b), nn, atol=4 * tol), (n, F)


def test_basis_is_the_natural_frame_at_the_pole():
    F = orc.make_basis([0.0, 0.0, 1.0])
    assert np.array_equal(np.abs(F), np.eye(3))
    assert np.array_equal(F, np.eye(3) + 0.0)
    # near the pole the frame moves continuously away from the natural one
    F = orc.make_basis(_unit([1e-4, -2e-4, 1.0]))
    assert np.allclose(F, np.eye(3), atol=5e-4)


# ----------------------------------------------------------------- SSAO: the frame in use

def _probe_kernel(dirs):
    k = np.zeros((len(dirs), 4), np.float32)
    k[:, :3] = dirs
    return k


@pytest.mark.parametrize("n", [(0.0, 0.0, 1.0), (0.6, 0.0, 0.8), (-0.3, 0.5, 0.81240384),
                               (0.7, -0.7, 0.14142136), (0.8, 0.3, -0.52), (-0.2, -0.9, -0.38729833)])
def test_ssao_tilted_normal_on_constant_depth(n):
    """Constant depth d everywhere and one tilted G-buffer normal n.  A sample
    S = P + r (k_x t + k_y b + k_z n) lands at view depth d - r (k . z) with
    z = (t_z, b_z, n_z); the buffer holds d at its pixel, so it is occluded exactly when
    r (k . z) <= -bias.  For any orthonormal frame z is a unit vector whose third entry is
    n_z, so a ring of in-plane directions at length l is occluded on an arc of half-angle
    arccos(bias / (r l sqrt(1 - n_z^2))) whatever the frame's rotation about n; directions
    along n are occluded when r l n_z <= -bias.  The exact set follows from the pinned
    frame."""
    n = _unit(n)
    H = W = 96
    d, r, bias = 2.5, 0.5, 0.0125
    normal = flat_normals(H, W, tuple(n))
    fr = synthetic_frame(np.full((H, W), d), normal)
    M = 720
    phi = 2 * math.pi * (np.arange(M) + 0.25) / M
    for ell in (1.0, 0.3, 0.1):
        ring = np.stack([ell * np.cos(phi), ell * np.sin(phi), np.zeros(M)], 1)
        cfg = orc.default_config("ssao", 4, samples=M, radius=r, ao_bias=bias, kernel=_probe_kernel(ring))
        for prec in ("f64", "f32"):
            ao = float(orc.shade_pixel(fr, cfg, W // 2, H // 2, prec)[0])
            occ = round((1 - ao) * M)
            rho = math.sqrt(max(0.0, 1 - n[2] ** 2))
            kappa = bias / (r * ell * rho) if rho > 0 else math.inf
            expect = M * math.acos(kappa) / math.pi if kappa < 1 else 0.0
            assert abs(occ - expect) <= 1.5, (n, ell, prec, occ, expect)
            # exact set with the frame itself
            zrow = orc.make_basis(n, "f64")[:, 2]
            disp = r * (ring @ zrow)
            lo, hi = int(np.sum(disp <= -bias - 1e-6)), int(np.sum(disp <= -bias + 1e-6))
            assert lo <= occ <= hi, (n, ell, prec, occ, lo, hi)
    # along the normal only
    for ell in (0.05, 0.5, 1.0):
        cfg = orc.default_config("ssao", 4, samples=1, radius=r, ao_bias=bias,
                                 kernel=_probe_kernel([[0.0, 0.0, ell]]))
        ao = float(orc.shade_pixel(fr, cfg, W // 2, H // 2, "f64")[0])
        assert ao == (0.0 if r * ell * n[2] <= -bias else 1.0), (n, ell, ao)


# ----------------------------------------------------------------- SSGI magnitude

def _pix_slopes(x, y, W, H, th=TAN30):
    """Ray slopes of the pixel centre (x, y) of a W x H pinhole image."""
    return ((x + 0.5) / W * 2 - 1) * th * W / H, (1 - (y + 0.5) / H * 2) * th


def _project(S, W, H, th=TAN30):
    dz = -S[2]
    return ((S[0] / dz) / (th * W / H) + 1) * W / 2, (1 - (S[1] / dz) / th) * H / 2


def _ssgi_case(n0, ell, ds_rel, r, N=1):
    """Shaded pixel p0 on a surface (depth 2, normal n0); one sample along n0 of length
    ell; its projected pixel s holds depth ds_rel * 2 and a normal facing back along the
    sample direction; colour (0.3, 0.5, 0.7) there.  Every other pixel is sky.  Returns
    the frame, the config and the expected GI from the pinhole definitions."""
    W, H = 64, 64
    x0, y0, d0 = 20, 30, 2.0
    n0 = _unit(n0)
    sx, sy = _pix_slopes(x0, y0, W, H)
    P = d0 * np.array([sx, sy, -1.0])
    S = P + r * ell * n0
    X, Y = _project(S, W, H)
    assert min(abs(X - round(X)), abs(Y - round(Y))) > 1e-3, "sample too close to a pixel border"
    ix, iy = int(math.floor(X)), int(math.floor(Y))
    assert (ix, iy) != (x0, y0)
    depth = np.full((H, W), 50.0)
    normal = np.zeros((H, W, 4))
    color = np.zeros((H, W, 4))
    depth[y0, x0] = d0
    normal[y0, x0, :3] = n0
    ds = d0 * ds_rel
    sxs, sys_ = _pix_slopes(ix, iy, W, H)
    Ps = ds * np.array([sxs, sys_, -1.0])
    D = Ps - P
    dd = float(D @ D)
    om = D / math.sqrt(dd)
    ns = _unit(-om + np.array([0.0, 0.2, 0.3]))
    depth[iy, ix] = ds
    normal[iy, ix, :3] = ns
    C = np.array([0.3, 0.5, 0.7])
    color[iy, ix, :3] = C
    fr = synthetic_frame(depth, normal, color)
    kern = [[0.0, 0.0, ell]]
    if N == 2:
        kern.append([0.0, 0.0, -ell])  # points into the surface: projects to sky, adds nothing
    dmin2 = (0.1 * r) ** 2
    cfg = orc.default_config("ssgi", 4, samples=N, radius=r, gi_min_dist2=dmin2, kernel=_probe_kernel(kern))
    if dd > r * r:
        return fr, cfg, np.zeros(3), dd, dmin2
    g = max(0.0, float(n0 @ om)) * max(0.0, float(-ns @ om)) / max(dd, dmin2)
    return fr, cfg, (r * r / N) * C * g, dd, dmin2


@pytest.mark.parametrize("N", [1, 2])
def test_ssgi_single_sample_form_factor_above_the_clamp(N):
    r = 0.6
    fr, cfg, expect, dd, dmin2 = _ssgi_case((0.3, 0.1, 0.9), 0.5, 0.9, r, N)
    assert dmin2 * 2 < dd < r * r
    got = orc.shade_pixel(fr, cfg, 20, 30, "f64")
    assert expect.min() > 0
    assert np.allclose(got, expect, rtol=2e-5, atol=0), (got, expect)
    got32 = orc.shade_pixel(fr, cfg, 20, 30, "f32")
    assert np.allclose(got32, expect, rtol=2e-4, atol=0)


def test_ssgi_single_sample_form_factor_below_the_clamp():
    r = 0.6
    fr, cfg, expect, dd, dmin2 = _ssgi_case((0.6, 0.0, 0.8), 0.1, 1.0, r)
    assert 0 < dd < dmin2 * 0.8
    got = orc.shade_pixel(fr, cfg, 20, 30, "f64")
    assert expect.min() > 0
    assert np.allclose(got, expect, rtol=2e-5, atol=0), (got, expect)


def test_ssgi_single_sample_out_of_range_adds_nothing():
    r = 0.6
    fr, cfg, expect, dd, _ = _ssgi_case((0.3, 0.1, 0.9), 0.9, 1.4, r)
    assert dd > r * r
    assert np.all(orc.shade_pixel(fr, cfg, 20, 30, "f64") == 0.0)


# ----------------------------------------------------------------- SSM shadow edges

def _light_frame(fr):
    """Receiver depth and shadow-map texel coordinates of every pixel, from the camera
    and light definitions (float64), as in a textbook shadow-map lookup."""
    cam, L = fr.cam, fr.light
    W, H = fr.width, fr.height
    d = fr.depth.astype(np.float64)
    th = float(cam.tan_half_fov)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    sx = ((x + 0.5) / W * 2.0 - 1.0) * th * (W / H)
    sy = (1.0 - (y + 0.5) / H * 2.0) * th
    e, rt, up, fw = (np.asarray(v, np.float64) for v in (cam.eye, cam.right, cam.up, cam.forward))
    world = e + (sx * d)[..., None] * rt + (sy * d)[..., None] * up + d[..., None] * fw
    rel = world - np.asarray(L.eye, np.float64)
    zr = rel @ np.asarray(L.forward, np.float64)
    ut = (rel @ np.asarray(L.right, np.float64)) / zr
    vt = (rel @ np.asarray(L.up, np.float64)) / zr
    tl = float(L.tan_half_fov)
    S = fr.shadow_map.shape[0]
    return zr, (ut + tl) * S / (2 * tl), (tl - vt) * S / (2 * tl)


def test_ssm_shadow_edges_follow_the_hard_shadow_boundary():
    W, H, S = 160, 120, 512
    fr = sg.gbuffer(0, W, H, 0, 0, shadow_size=S)       # ground plane only
    zb = 6.0
    sm = np.full((S, S), sg.LIGHT_FAR, np.float32)
    sm[:, : S // 2] = zb                                   # a half-plane occluder
    fr.shadow_map = sm
    cfg = orc.default_config("ssm", 4, kernel=sg.hemisphere_kernel(16),
                             blocker_taps=sg.disk_taps(32, sg.BLOCKER_SEED), pcf_taps=sg.disk_taps(64, sg.PCF_SEED))
    bias = cfg["shadow_bias"]
    zr, Xt, Yt = _light_frame(fr)
    sky = fr.depth >= fr.cam.far
    on_map = (Xt >= 0) & (Xt < S) & (Yt >= 0) & (Yt < S)
    shadowed = on_map & (np.floor(Xt) < S // 2) & (zb < zr - bias)
    hs_ref = np.where(shadowed, 0, 1)
    # pixels whose lookup sits within rounding of a decision boundary are left open
    unsure = (np.abs(Xt - S // 2) < 1e-3) | (np.abs(Xt) < 1e-3) | (np.abs(Xt - S) < 1e-3) | \
             (np.abs(Yt) < 1e-3) | (np.abs(Yt - S) < 1e-3) | (np.abs(zr - bias - zb) < 1e-4)
    unsure &= ~sky
    hs = orc.hard_shadow(fr, cfg, "f64")
    ok = ~sky & ~unsure
    assert np.array_equal(hs[ok], hs_ref[ok])
    assert (hs_ref[ok] == 0).sum() > 500 and (hs_ref[ok] == 1).sum() > 500
    # expected shadow edges: a 4-neighbour (in the image, not sky) with another hard shadow
    exp = np.zeros((H, W), bool)
    near_unsure = unsure.copy()
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        a = np.zeros((H, W), bool)
        u = np.zeros((H, W), bool)
        ys = slice(max(0, -dy), H - max(0, dy))
        yd = slice(max(0, dy), H - max(0, -dy))
        xs = slice(max(0, -dx), W - max(0, dx))
        xd = slice(max(0, dx), W - max(0, -dx))
        a[ys, xs] = (hs_ref[yd, xd] != hs_ref[ys, xs]) & ~sky[yd, xd]
        u[ys, xs] = unsure[yd, xd]
        exp |= a
        near_unsure |= u
    exp &= ~sky
    geo = orc.edges(fr, orc.default_config("ssao", 4), "f64").astype(bool)
    for prec in ("f64", "f32"):
        E = orc.edges(fr, cfg, prec).astype(bool)
        keep = ~near_unsure
        assert np.array_equal(E[keep], (geo | exp)[keep]), prec
    assert (exp & ~geo & ~near_unsure).sum() > 80           # the boundary crosses the view
