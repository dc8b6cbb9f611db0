"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
an invariant, a brute-force restatement in a different form, or a library routine.
Paper citations are to arXiv 1906.04576.
"""
import math

import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from conftest import flat_normals, synthetic_frame

TAN30 = math.tan(math.radians(30.0))


def cfg_for(effect="ssao", levels=4, **kw):
    kw.setdefault("kernel", sg.hemisphere_kernel(kw.get("samples", 16)))
    return orc.default_config(effect, levels, **kw)


# ----------------------------------------------------------------- level geometry

def test_level_dims_match_the_paper_resolutions():
    # Sec. 4: widths halved -- full, 1/2, 1/4, 1/8 of 1920x1080, 2560x1440, 3840x2160.
    for (W, H) in [(1920, 1080), (2560, 1440), (3840, 2160), (256, 256)]:
        for i in range(4):
            assert orc.level_dim(W, i) == W // (1 << i)
            assert orc.level_dim(H, i) == H // (1 << i)
    # ragged sizes: every pixel belongs to a block of every level
    for n in (1, 2, 7, 257, 1001):
        for i in range(4):
            assert orc.level_dim(n, i) == -(-n // (1 << i))
            assert (n - 1) >> i < orc.level_dim(n, i)


def test_level_sample_is_block_centre_clamped():
    for i in range(4):
        for q in range(0, 40):
            s = orc.level_sample(q, i, 100)
            assert s == min(q * (1 << i) + (0 if i == 0 else (1 << (i - 1))), 99)
            if s < 99:
                assert q * (1 << i) <= s < (q + 1) * (1 << i)


# ----------------------------------------------------------------- binary16 rounding

def test_round_to_half_matches_numpy_float16():
    rng = np.random.default_rng(1)
    vals = np.concatenate([
        rng.standard_normal(4000).astype(np.float32),
        (rng.random(2000) * 1e-4).astype(np.float32),   # subnormal half range
        (rng.random(1000) * 7e4).astype(np.float32),    # around overflow
        np.array([0.0, -0.0, 1.0, 65504.0, 65519.0, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                  1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -14], np.float32),
    ])
    ours = np.array([orc.round_to_half(float(v)) for v in vals], np.float32)
    with np.errstate(over="ignore"):
        ref = vals.astype(np.float16).astype(np.float32)
    assert np.array_equal(ours, ref, equal_nan=True)


# ----------------------------------------------------------------- Gaussian weights

@pytest.mark.parametrize("sigma2,R", [(0.924, 3), (1.848, 5), (3.696, 6)])
def test_gauss_weights_radius_symmetry_normalisation(sigma2, R):
    g64 = orc.gauss_weights(sigma2, np.float64)
    g32 = orc.gauss_weights(sigma2, np.float32)
    assert len(g64) == 2 * R + 1 == len(g32)
    assert R == math.ceil(3.0 * math.sqrt(sigma2))
    assert abs(g64.sum() - 1.0) < 1e-15
    assert np.array_equal(g32, g32[::-1]) and np.array_equal(g64, g64[::-1])
    # ratio of neighbouring taps of a Gaussian: exp(-(2k+1) / (2 sigma^2))
    for k in range(R):
        assert math.isclose(g64[R + k + 1] / g64[R + k], math.exp(-(2 * k + 1) / (2 * sigma2)), rel_tol=1e-12)
    assert np.all(g32 > 0)


# ----------------------------------------------------------------- view reconstruction

def test_view_position_reconstructs_the_ray_cast_hit_point():
    """P(x, y, d) mapped to world space equals the generator's own hit point."""
    W, H = 96, 64
    fr = sg.gbuffer(3, W, H, 8, 4)
    cfg = cfg_for()
    cam = fr.cam
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(200):
        x, y = int(rng.integers(W)), int(rng.integers(H))
        d = float(fr.depth[y, x])
        hit = sg.pixel_world(3, W, H, 8, 4, x, y)
        if hit is None:
            assert d == cam.far
            continue
        P = orc.view_pos(fr, cfg, x, y, d, "f64")
        world = (cam.eye.astype(np.float64) + P[0] * cam.right + P[1] * cam.up - P[2] * cam.forward)
        assert np.allclose(world, hit, rtol=0, atol=2e-5 * d), (x, y, world, hit)
        checked += 1
    assert checked > 100


# ----------------------------------------------------------------- edges (Sec. 3.1)

def _edges(depth, normal, **kw):
    fr = synthetic_frame(depth, normal)
    return orc.edges(fr, cfg_for(**kw))


def test_flat_and_tilted_planes_have_no_edges():
    H, W = 24, 32
    assert _edges(np.full((H, W), 3.0), flat_normals(H, W)).sum() == 0
    ramp = 2.0 + 0.01 * np.arange(W)[None, :] + 0.02 * np.arange(H)[:, None]
    assert _edges(np.broadcast_to(ramp, (H, W)), flat_normals(H, W)).sum() == 0


def test_depth_step_marks_both_sides_only():
    H, W = 16, 32
    d = np.full((H, W), 2.0)
    d[:, 16:] = 3.0
    E = _edges(d, flat_normals(H, W))
    expect = np.zeros((H, W), np.uint8)
    expect[:, 15:17] = 1
    assert np.array_equal(E, expect)


def test_depth_second_difference_threshold_is_relative():
    # second difference 2*delta at the kink pixel; threshold 0.05 * depth
    H, W = 8, 20
    for delta, hit in [(0.04, False), (0.06, True)]:
        d = np.full((H, W), 2.0)
        d[:, 10] = 2.0 + delta   # spike: |lap| = 2 delta at x=10, delta at x=9 and 11
        E = _edges(d, flat_normals(H, W))
        # at x=10: |lap| = 2 delta vs 0.05 * (2 + delta)
        assert bool(E[4, 10]) == (2 * delta > 0.05 * (2 + delta))
        assert bool(E[4, 9]) == (delta > 0.05 * 2.0) == bool(E[4, 11])
        assert hit == bool(E[4, 10])


def test_normal_crease_threshold():
    H, W = 8, 16
    for n2, hit in [((0.6, 0.0, 0.8), True), ((0.3, 0.0, math.sqrt(0.91)), False)]:
        n = flat_normals(H, W)
        n[:, 8:, 0], n[:, 8:, 1], n[:, 8:, 2] = n2
        E = _edges(np.full((H, W), 3.0), n)
        expect = np.zeros((H, W), np.uint8)
        if hit:
            expect[:, 7:9] = 1
        assert np.array_equal(E, expect)


def test_sky_is_never_an_edge_and_its_neighbours_are():
    H, W = 12, 12
    d = np.full((H, W), 3.0)
    d[:4, :] = 50.0   # sky (= far)
    n = flat_normals(H, W)
    n[:4] = 0
    E = _edges(d, n)
    assert E[:4].sum() == 0
    assert np.all(E[4] == 1)
    assert E[5:].sum() == 0


def test_image_border_does_not_make_edges():
    H, W = 10, 10
    d = np.full((H, W), 2.0)
    d[:, 0] = 5.0     # a step right at the border: the x-axis test is skipped at x=0
    E = _edges(d, flat_normals(H, W))
    assert np.all(E[:, 1] == 1)          # x=1 sees the step
    assert np.all(E[:, 0] == 0)          # x=0 has no left neighbour: no second difference
    assert E[:, 2:].sum() == 0


# ----------------------------------------------------------------- masks (Sec. 3.1, Table 1)

def _masks_from_E(E, levels=4, effect="ssao", **kw):
    H, W = E.shape
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for(effect, levels, **kw)
    return cfg, orc.masks(fr, cfg, E.astype(np.uint8))


def test_single_edge_pixel_gives_square_regions():
    """One edge texel: S_0 is the (2R_0+1)^2 square, a_0 the outer product of g."""
    H, W = 64, 64
    E = np.zeros((H, W), np.uint8)
    E[30, 21] = 1
    cfg, (a, S, label) = _masks_from_E(E)
    g0 = orc.gauss_weights(0.924, np.float64)
    R0 = len(g0) // 2
    expect = np.zeros((H, W), bool)
    expect[30 - R0:31 + R0, 21 - R0:22 + R0] = True
    assert np.array_equal(S[0].astype(bool), expect)
    outer = np.zeros((H, W))
    outer[30 - R0:31 + R0, 21 - R0:22 + R0] = np.outer(g0, g0)
    assert np.allclose(a[0], outer, rtol=1e-6, atol=0)
    # level 1: block (15, 10) dilated by R_1 = 5, plus the parents of S_0
    R1 = len(orc.gauss_weights(1.848)) // 2
    e1 = np.zeros(S[1].shape, bool)
    e1[15 - R1:16 + R1, 10 - R1:11 + R1] = True
    ys, xs = np.nonzero(S[0])
    e1[ys >> 1, xs >> 1] = True
    assert np.array_equal(S[1].astype(bool), e1)
    assert np.all(S[3] == 1) and np.all(a[3] == 1)
    # labels: 0 inside the level-0 square
    assert np.all(label[expect] == 0)


def test_masks_brute_force_2d_gaussian_8x8():
    """Separable FP32 blur vs a direct 2-D double Gaussian sum on random 8x8 edge images."""
    rng = np.random.default_rng(7)
    for trial in range(40):
        E = (rng.random((8, 8)) < rng.uniform(0.02, 0.3)).astype(np.uint8)
        cfg, (a, S, label) = _masks_from_E(E, levels=3)
        for i, s2 in enumerate(cfg["sigma2"][:2]):
            Wi = 8 >> i
            D = E.reshape(Wi, 1 << i, Wi, 1 << i).max(axis=(1, 3))
            R = math.ceil(3 * math.sqrt(s2))
            ks = np.arange(-R, R + 1)
            g = np.exp(-ks ** 2 / (2 * s2))
            g /= g.sum()
            ref = np.zeros((Wi, Wi))
            for y in range(Wi):
                for x in range(Wi):
                    for dy in range(-R, R + 1):
                        for dx in range(-R, R + 1):
                            yy, xx = y + dy, x + dx
                            if 0 <= yy < Wi and 0 <= xx < Wi:
                                ref[y, x] += g[dy + R] * g[dx + R] * D[yy, xx]
            assert np.allclose(a[i], ref, rtol=2e-6, atol=1e-12)
            raw = ref > 0
            if i == 0:
                assert np.array_equal(S[0].astype(bool), raw)
            else:
                prev = np.zeros_like(raw)
                ys, xs = np.nonzero(S[i - 1])
                prev[ys >> 1, xs >> 1] = True
                assert np.array_equal(S[i].astype(bool), raw | prev)
        # label: every pixel exactly one level, the finest whose stencil covers it
        for y in range(8):
            for x in range(8):
                covering = [i for i in range(3) if S[i][y >> i, x >> i]]
                assert label[y, x] == min(covering)


@pytest.mark.parametrize("effect", ["ssao", "ssgi"])
def test_masks_partition_and_nesting_on_scenes(effect):
    fr = sg.gbuffer(11, 203, 141, 16, 6)      # ragged size
    cfg = cfg_for(effect, 4)
    E = orc.edges(fr, cfg)
    a, S, label = orc.masks(fr, cfg, E)
    enabled = [i for i in range(4) if cfg["enabled"][i]]
    assert set(np.unique(label)) <= set(enabled)
    assert np.all(S[3] == 1)
    for i, j in zip(enabled, enabled[1:]):
        f = 1 << (j - i)
        ys, xs = np.nonzero(S[i])
        assert np.all(S[j][ys // f, xs // f] == 1)        # inclusion of finer areas
    for i in range(4):
        assert np.all((a[i] >= 0) & (a[i] <= 1 + 1e-6))
        if cfg["enabled"][i] and i < 3:
            assert np.all(S[i][a[i] > 0] == 1)           # stencil = [mask > 0] (Sec. 4.1)
        if not cfg["enabled"][i]:
            assert S[i].sum() == 0
    # every pixel's label level has its stencil set, and no finer enabled level does
    H, W = label.shape
    yy, xx = np.mgrid[0:H, 0:W]
    for i in enabled:
        set_i = S[i][yy >> i, xx >> i].astype(bool)
        assert np.all(set_i[label == i])
        assert not np.any(set_i[label > i])


def test_compaction_is_row_major_nonzero():
    rng = np.random.default_rng(3)
    S = (rng.random((37, 53)) < 0.3).astype(np.uint8)
    wl = orc.compact(S)
    ys, xs = np.nonzero(S)
    assert np.array_equal(wl, (ys.astype(np.uint32) << 16) | xs.astype(np.uint32))


# ----------------------------------------------------------------- SSAO (Sec. 2.4)

def test_ssao_fronto_parallel_plane_is_unoccluded():
    H, W = 48, 64
    fr = synthetic_frame(np.full((H, W), 2.5), flat_normals(H, W))
    cfg = cfg_for(samples=64)
    for prec in ("f32", "f64"):
        assert np.all(orc.shade_full(fr, cfg, prec) == 1.0)


def _step_scene(d_near, d_far):
    H = W = 64
    d = np.full((H, W), d_far)
    d[:, :32] = d_near
    return synthetic_frame(d, flat_normals(H, W))


def test_ssao_depth_step_closed_form():
    """Far plane next to a nearer half-plane: a sample is occluded exactly when it
    projects onto the near half and sits behind it by more than the bias."""
    N, r, bias = 64, 0.5, 0.0125
    d1, d2 = 2.0, 2.2
    fr = _step_scene(d1, d2)
    cfg = cfg_for(samples=N, radius=r, ao_bias=bias)
    k = cfg["kernel"].astype(np.float64)
    total = 0
    for (x, y) in [(32, 5), (33, 20), (34, 40), (36, 10), (40, 33)]:
        # pinhole geometry with the textbook tangent of 30 degrees
        px = ((x + 0.5) / 32.0 - 1.0) * TAN30 * d2
        py = (1.0 - (y + 0.5) / 32.0) * TAN30 * d2
        lo = hi = 0
        for j in range(N):
            sx, sy, depth_s = px + r * k[j, 0], py + r * k[j, 1], d2 - r * k[j, 2]
            col = 32.0 + 32.0 * sx / (depth_s * TAN30)
            row = 32.0 - 32.0 * sy / (depth_s * TAN30)
            behind = d1 - (depth_s - bias)           # <= 0: occluded by the near plane
            if not (0 <= row < 64) or col >= 32 + 1e-4 or behind > 1e-5:
                continue
            hi += 1
            if col < 32 - 1e-4 and behind < -1e-5:
                lo += 1
        ao = orc.shade_pixel(fr, cfg, x, y, "f32")[0]
        occ = round((1.0 - ao) * N)
        assert lo <= occ <= hi, (x, y, occ, lo, hi)
        total += lo
    assert total > 0
    # the near plane itself sees nothing in front of it
    for (x, y) in [(30, 20), (10, 40)]:
        assert orc.shade_pixel(fr, cfg, x, y, "f32")[0] == 1.0


def test_ssao_range_check_ignores_distant_occluders():
    # depth gap 1.0 > r = 0.5: the near half-plane is out of range
    fr = _step_scene(2.0, 3.0)
    cfg = cfg_for(samples=64, radius=0.5)
    assert np.all(orc.shade_full(fr, cfg)[:, 32:] == 1.0)


def test_ssao_sky_is_one_and_bounds():
    fr = sg.gbuffer(5, 160, 90, 12, 4)
    cfg = cfg_for(samples=32)
    ao = orc.shade_full(fr, cfg)[..., 0]
    assert np.all(ao[fr.depth >= fr.cam.far] == 1.0)
    assert np.all((ao >= 0) & (ao <= 1))
    # values are multiples of 1/N
    assert np.allclose(np.round(ao * 32), ao * 32, atol=1e-5)
    assert ao.min() < 0.9      # the scene has creases


# ----------------------------------------------------------------- SSGI (Sec. 2.4)

def test_ssgi_flat_plane_is_zero_and_linear_in_color():
    H, W = 40, 40
    col = np.ones((H, W, 4), np.float32)
    fr = synthetic_frame(np.full((H, W), 2.0), flat_normals(H, W), col)
    cfg = cfg_for("ssgi", samples=32, radius=1.0)
    assert np.all(orc.shade_full(fr, cfg) == 0.0)
    # a real scene: GI is linear in the direct light (x2 is exact in binary floating point)
    fr = sg.gbuffer(2, 96, 64, 12, 4)
    g1 = orc.shade_full(fr, cfg, "f64")
    fr.color = fr.color * 2
    g2 = orc.shade_full(fr, cfg, "f64")
    assert np.array_equal(g2, 2 * g1)
    assert g1.max() > 0
    fr.color[:] = 0
    assert np.all(orc.shade_full(fr, cfg) == 0)


def test_ssgi_facing_walls_receive_light():
    """Left half: a wall facing +x; right half: a wall facing -x (a V seen from the front)."""
    H, W = 32, 64
    d = np.full((H, W), 2.0)
    n = flat_normals(H, W)
    s = math.sqrt(0.5)
    n[:, :32, 0], n[:, :32, 2] = s, s      # faces right (+x) and toward the camera
    n[:, 32:, 0], n[:, 32:, 2] = -s, s     # faces left
    # depth consistent with the V: deeper toward the middle
    x = np.arange(W)
    d = 2.0 + 0.02 * (32 - np.abs(x - 31.5))[None, :] * np.ones((H, 1))
    col = np.zeros((H, W, 4), np.float32)
    col[:, 32:, 0] = 1.0                    # only the right wall is lit, red
    fr = synthetic_frame(d, n, col)
    cfg = cfg_for("ssgi", samples=64, radius=1.0)
    gi = orc.shade_full(fr, cfg, "f64")
    assert gi[16, 28, 0] > 0               # left wall next to the crease receives red
    assert np.all(gi[..., 1:] == 0)         # no green or blue anywhere
    assert np.all(gi >= 0)


# ----------------------------------------------------------------- SSM (Sec. 2.4)

def _ssm_frame(sm_value, W=64, H=48):
    fr = sg.gbuffer(0, W, H, 0, 0, shadow_size=256)   # ground plane only
    fr.shadow_map = np.full((256, 256), sm_value, np.float32)
    return fr


def _ssm_cfg():
    return cfg_for("ssm", blocker_taps=sg.disk_taps(32, sg.BLOCKER_SEED),
                   pcf_taps=sg.disk_taps(64, sg.PCF_SEED))


def test_ssm_no_blocker_is_lit_and_full_umbra_is_zero():
    cfg = _ssm_cfg()
    fr = _ssm_frame(sg.LIGHT_FAR)                     # nothing between light and scene
    vis = orc.shade_full(fr, cfg)[..., 0]
    assert np.all(vis == 1.0)
    fr = _ssm_frame(sg.LIGHT_NEAR + 0.5)              # an occluder covering the whole map
    vis = orc.shade_full(fr, cfg)[..., 0]
    ground = fr.depth < fr.cam.far
    # off-map taps are lit by definition, so only the lower half of the view (the ground
    # near the origin, deep inside the light's frustum) is a full umbra
    H, W = vis.shape
    assert np.all(vis[H // 2:] == 0.0)
    assert np.all(vis[~ground] == 1.0)
    hs = orc.hard_shadow(fr, cfg)
    assert np.all(hs[H // 2:] == 0)


def test_ssm_ground_only_scene_is_lit():
    fr = sg.gbuffer(0, 80, 60, 0, 0, shadow_size=512)
    vis = orc.shade_full(fr, _ssm_cfg(), "f64")[..., 0]
    assert np.all(vis == 1.0)


def test_ssm_box_casts_umbra_and_penumbra():
    fr = sg.gbuffer(4, 160, 120, 8, 0, shadow_size=1024)
    cfg = _ssm_cfg()
    vis = orc.shade_full(fr, cfg, "f64")[..., 0]
    hs = orc.hard_shadow(fr, cfg, "f64")
    ground = fr.objid == 0
    assert (vis[ground] == 0).any() and (vis[ground] == 1).any()
    soft = (vis > 0) & (vis < 1)
    assert soft.any()
    # the hard shadow of one sample agrees with PCSS in umbra and fully lit regions
    assert np.all(hs[ground & (vis == 0)] == 0)
    assert np.mean(hs[ground & (vis == 1)] == 1) > 0.99


def test_ssm_penumbra_width_follows_similar_triangles():
    """A half-plane occluder at light depth z_b over the ground (the left half of the
    shadow map; its edge is the map's middle column, tangent coordinate 0).  PCSS must
    leave a ground point fully dark or fully lit outside a band around the edge whose
    half-width, in the light's tangent units at receiver depth z_r, is
    R = (l/2)(z_r - z_b)/(z_b z_r) -- Fernando's similar triangles: a penumbra of world
    width l (z_r - z_b)/z_b on the receiver -- and partly lit in the inner third of the
    band.  Receiver positions come from the pinhole definitions here, not from the oracle."""
    W, H, S = 160, 120, 512
    fr = sg.gbuffer(0, W, H, 0, 0, shadow_size=S)        # ground plane only
    zb, l = 6.0, 0.5
    sm = np.full((S, S), sg.LIGHT_FAR, np.float32)
    sm[:, : S // 2] = zb
    fr.shadow_map = sm
    cfg = _ssm_cfg()
    assert cfg["light_size"] == l
    vis = orc.shade_full(fr, cfg, "f64")[..., 0]
    cam, L = fr.cam, fr.light
    d = fr.depth.astype(np.float64)
    th = float(cam.tan_half_fov)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    sx = ((x + 0.5) / W * 2.0 - 1.0) * th * (W / H)
    sy = (1.0 - (y + 0.5) / H * 2.0) * th
    e, r, u, f = (np.asarray(v, np.float64) for v in (cam.eye, cam.right, cam.up, cam.forward))
    world = e + (sx * d)[..., None] * r + (sy * d)[..., None] * u + d[..., None] * f
    rel = world - np.asarray(L.eye, np.float64)
    zr = rel @ np.asarray(L.forward, np.float64)
    ut = (rel @ np.asarray(L.right, np.float64)) / zr
    vt = (rel @ np.asarray(L.up, np.float64)) / zr
    R = (l / 2) * (zr - zb) / (zb * zr)
    tl = float(L.tan_half_fov)
    ground = (fr.depth < cam.far) & (np.abs(ut) < 0.8 * tl) & (np.abs(vt) < 0.8 * tl)
    dark = ground & (ut < -R * (1 + 1e-3))
    lit = ground & (ut > R * (1 + 1e-3))
    inner = ground & (np.abs(ut) < R / 3)
    assert dark.sum() > 100 and lit.sum() > 100 and inner.sum() > 10
    assert np.all(vis[dark] == 0.0)
    assert np.all(vis[lit] == 1.0)
    assert np.all((vis[inner] > 0.0) & (vis[inner] < 1.0))
    # the band is really as wide as the formula: halving it would misclassify pixels
    assert np.any((vis > 0) & (vis < 1) & ground & (np.abs(ut) > R / 2))


# ----------------------------------------------------------------- blending (Sec. 4.2, Eq. 1)

def _levels_like(H, W, L, fill):
    return [np.full((orc.level_dim(H, i), orc.level_dim(W, i), 1), fill, np.float32) for i in range(L)]


def test_constant_subimages_survive_upsample_and_merge():
    rng = np.random.default_rng(5)
    H, W, L = 45, 67, 4
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for("ssao", L)
    E = (rng.random((H, W)) < 0.02).astype(np.uint8)
    a, S, _ = orc.masks(fr, cfg, E)
    for K in (0.3, 0.7779, 1.0):
        c = _levels_like(H, W, L, K)
        for i in range(L):
            c[i][S[i] == 0] = np.nan          # unrendered texels are never read
        out = orc.merge(fr, cfg, a, S, c)
        assert np.all(np.isfinite(out))
        assert np.allclose(out, K, rtol=4e-7, atol=0)


def test_bilinear_reproduces_linear_ramps_at_sample_positions():
    """Two levels, the coarsest alone visible: c_1(q) = x of its sample pixel gives
    c'(p) = p_x away from the clamped borders (pins origin o_1 and scale 2)."""
    H, W = 20, 40
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for("ssao", 2, enabled=[1, 1, 0, 0], weight=[0.0, 1.0, 0, 0])
    a = [np.zeros((H, W), np.float32), np.ones((H // 2, W // 2), np.float32)]
    S = [np.zeros((H, W), np.uint8), np.ones((H // 2, W // 2), np.uint8)]
    qx = np.arange(W // 2)
    c1 = np.broadcast_to((2 * qx + 1).astype(np.float32)[None, :, None], (H // 2, W // 2, 1)).copy()
    c = [np.zeros((H, W, 1), np.float32), c1]
    out = orc.merge(fr, cfg, a, S, c)[..., 0]
    assert np.array_equal(out[:, 1:W - 1], np.broadcast_to(np.arange(1, W - 1, dtype=np.float32), (H, W - 2)))


def test_eq1_two_level_blend_closed_form():
    H, W = 16, 16
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for("ssao", 2, enabled=[1, 1, 0, 0], weight=[4.0, 1.0, 0, 0])
    A, B = 0.25, 0.75
    for a0 in (0.0, 0.05, 0.2, 0.3, 1.0):
        a = [np.full((H, W), a0, np.float32), np.ones((8, 8), np.float32)]
        S = [np.ones((H, W), np.uint8), np.ones((8, 8), np.uint8)]
        c = [np.full((H, W, 1), A, np.float32), np.full((8, 8, 1), B, np.float32)]
        out = orc.merge(fr, cfg, a, S, c, "f64")
        alpha = min(4.0 * float(np.float32(a0)), 1.0)
        assert np.allclose(out, A * alpha + B * (1 - alpha), rtol=1e-12, atol=1e-12)
        if alpha == 1.0:
            assert np.all(out == A)            # alpha = 1 returns c_i
        if alpha == 0.0:
            assert np.all(out == B)            # alpha = 0 returns the coarser composite


def test_masked_bilinear_ignores_unrendered_taps():
    H, W = 16, 16
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for("ssao", 2, enabled=[1, 1, 0, 0], weight=[1.0, 1.0, 0, 0])
    a = [np.zeros((H, W), np.float32), np.ones((8, 8), np.float32)]
    S1 = np.ones((8, 8), np.uint8)
    S1[:, 4:] = 0
    c1 = np.full((8, 8, 1), 0.5, np.float32)
    c1[:, 4:] = np.nan
    # the coarsest level is fully rendered by definition; use level 0 as the masked one
    a = [np.ones((H, W), np.float32), np.ones((8, 8), np.float32)]
    S0 = np.ones((H, W), np.uint8)
    S0[:, 8:] = 0
    c0 = np.full((H, W, 1), 0.25, np.float32)
    c0[:, 8:] = np.nan
    a[0][:, 8:] = 0
    out = orc.merge(fr, cfg, a, [S0, np.ones((8, 8), np.uint8)],
                    [c0, np.full((8, 8, 1), 0.75, np.float32)])
    assert np.all(np.isfinite(out))
    assert np.all(out[:, :8] == 0.25)
    assert np.all(out[:, 8:] == 0.75)


# ----------------------------------------------------------------- step-wise blending (Sec. 3.3)

def _stepwise_cfg(levels, **kw):
    return cfg_for("ssao", levels, merge_mode=1, **kw)


def test_stepwise_constant_subimages_survive():
    rng = np.random.default_rng(8)
    H, W, L = 45, 67, 4
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = _stepwise_cfg(L)
    E = (rng.random((H, W)) < 0.02).astype(np.uint8)
    a, S, _ = orc.masks(fr, cfg, E)
    for K in (0.3, 0.7779, 1.0):
        c = _levels_like(H, W, L, K)
        for i in range(L):
            c[i][S[i] == 0] = np.nan          # unrendered texels are never read
        for prec in ("f32", "f64"):
            out = orc.merge(fr, cfg, a, S, c, prec)
            assert np.all(np.isfinite(out))
            assert np.allclose(out, K, rtol=4e-7, atol=0)


@pytest.mark.parametrize("enabled", [[1, 1, 1, 0], [1, 0, 1, 1]])
def test_stepwise_chain_reproduces_linear_ramps(enabled):
    """Only the coarsest level visible (every other alpha 0): c(Q) = x of Q's sample pixel
    at the coarsest level is carried through each step (2x, or 4x over a disabled level)
    to c'(p) = p_x away from the clamped borders -- pins every step's origin and scale."""
    L = 3 if enabled[3] == 0 else 4
    H, W = 64, 96
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = _stepwise_cfg(L, enabled=enabled)
    a = [np.zeros((orc.level_dim(H, i), orc.level_dim(W, i)), np.float64) for i in range(L)]
    S = [np.zeros_like(x, dtype=np.uint8) for x in a]
    c = [np.full(x.shape + (1,), np.nan) for x in a]
    top = L - 1
    S[top][:] = 1
    qx = np.arange(orc.level_dim(W, top))
    c[top][:] = ((qx << top) + (1 << (top - 1))).astype(np.float64)[None, :, None]
    out = orc.merge(fr, cfg, a, S, c, "f64")[..., 0]
    m = 1 << (top + 1)
    assert np.array_equal(out[:, m:W - m], np.broadcast_to(np.arange(m, W - m, dtype=np.float64), (H, W - 2 * m)))


def test_stepwise_alpha_saturates_at_level_resolution():
    """Three levels; level 1 (w = 50) holds one rendered texel Q with a_1 = 0.04 and c = 1,
    the coarsest level is 0, level 0 is empty.  The chain saturates alpha at Q itself
    (min(50 * 0.04, 1) = 1, so c'_1(Q) = 1) and then interpolates: the pixel half-way to
    the next texel reads 1/2.  The direct merge interpolates a first (0.02, saturating
    to alpha = 1) and reads 1 there."""
    H, W = 32, 32
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    Q = (6, 5)                                  # (row, column) of level 1
    a = [np.zeros((H, W)), np.zeros((16, 16)), np.zeros((8, 8))]
    S = [np.zeros((H, W), np.uint8), np.zeros((16, 16), np.uint8), np.ones((8, 8), np.uint8)]
    c = [np.full((H, W, 1), np.nan), np.full((16, 16, 1), np.nan), np.zeros((8, 8, 1))]
    a[1][Q] = 0.04
    S[1][Q] = 1
    c[1][Q] = 1.0
    y, x = 2 * Q[0] + 1, 2 * Q[1] + 2           # level-1 coordinate (Q_row, Q_col + 1/2)
    step = orc.merge(fr, _stepwise_cfg(3), a, S, c, "f64")[..., 0]
    direct = orc.merge(fr, cfg_for("ssao", 3), a, S, c, "f64")[..., 0]
    assert step[y, x - 1] == 1.0 and step[y, x] == 0.5
    assert direct[y, x - 1] == 1.0 and direct[y, x] == 1.0
    # in the linear regime (no saturation) the two readings agree
    a[1][Q] = 0.01
    step = orc.merge(fr, _stepwise_cfg(3), a, S, c, "f64")[..., 0]
    direct = orc.merge(fr, cfg_for("ssao", 3), a, S, c, "f64")[..., 0]
    assert step[y, x] == 0.25 and direct[y, x] == 0.25


def test_stepwise_two_levels_is_eq1():
    H, W = 16, 16
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = _stepwise_cfg(2, enabled=[1, 1, 0, 0], weight=[4.0, 1.0, 0, 0])
    A, B = 0.25, 0.75
    for a0 in (0.0, 0.05, 0.2, 0.3, 1.0):
        a = [np.full((H, W), a0), np.ones((8, 8))]
        S = [np.ones((H, W), np.uint8), np.ones((8, 8), np.uint8)]
        c = [np.full((H, W, 1), A), np.full((8, 8, 1), B)]
        out = orc.merge(fr, cfg, a, S, c, "f64")
        alpha = min(4.0 * a0, 1.0)
        assert np.allclose(out, A * alpha + B * (1 - alpha), rtol=1e-12, atol=1e-12)


def test_stepwise_render_error_against_full_resolution_is_small():
    fr = sg.gbuffer(0, 256, 256, 8, 0)
    cfg = cfg_for("ssao", 3, samples=16, merge_mode=1)
    res = orc.render(fr, cfg)
    full = orc.shade_full(fr, cfg)
    assert float(np.sqrt(np.mean((res["out"] - full) ** 2))) <= 1e-2


def test_bilateral_merge_keeps_taps_on_the_pixels_surface():
    """Two levels, level 0 invisible (w_0 = 0): the output is the level-1 interpolation.
    Texels left of column k hold 0 at depth 1, the others 1 at depth 2 (their sample
    pixels 2q + 1 carry the depths).  Pixel 2k, half-way between texels k - 1 and k and at
    depth 2, reads 1/2 through the plain taps and 1 through the bilateral ones (the tap at
    depth 1 fails the depth test); on flat depth both readings agree exactly, and where no
    tap passes the bilateral reading falls back to the plain one."""
    H, W, k = 16, 32, 7
    depth = np.full((H, W), 1.0)
    depth[:, 2 * k:] = 2.0
    fr = synthetic_frame(depth, flat_normals(H, W))
    kw = dict(enabled=[1, 1, 0, 0], weight=[0.0, 1.0, 0, 0], blur_depth_rel=0.05)
    a = [np.zeros((H, W)), np.ones((8, 16))]
    S = [np.zeros((H, W), np.uint8), np.ones((8, 16), np.uint8)]
    c1 = np.zeros((8, 16, 1))
    c1[:, k:] = 1.0
    c = [np.full((H, W, 1), np.nan), c1]
    bil = orc.merge(fr, cfg_for("ssao", 2, merge_mode=2, **kw), a, S, c, "f64")[..., 0]
    plain = orc.merge(fr, cfg_for("ssao", 2, **kw), a, S, c, "f64")[..., 0]
    assert np.all(plain[:, 2 * k] == 0.5) and np.all(bil[:, 2 * k] == 1.0)
    assert np.all(bil[:, : 2 * k] == 0.0) and np.all(bil[:, 2 * k:] == 1.0)
    flat = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    for cc in (c, [np.full((H, W, 1), np.nan), np.random.default_rng(1).random((8, 16, 1))]):
        assert np.array_equal(orc.merge(flat, cfg_for("ssao", 2, merge_mode=2, **kw), a, S, cc, "f64"),
                              orc.merge(flat, cfg_for("ssao", 2, **kw), a, S, cc, "f64"))
    # a pixel whose depth matches no tap (a thin sliver at depth 9) falls back to the plain taps
    sliver = depth.copy()
    sliver[:, 2 * k] = 9.0
    fr2 = synthetic_frame(sliver, flat_normals(H, W))
    bil2 = orc.merge(fr2, cfg_for("ssao", 2, merge_mode=2, **kw), a, S, c, "f64")[..., 0]
    assert np.all(bil2[:, 2 * k] == 0.5)


# ----------------------------------------------------------------- sample-count levels (Sec. 6)

def test_sample_levels_shade_blocks_of_listed_texels_with_thinned_tables():
    """Level i >= 1 shades every pixel of each listed texel's 2^i x 2^i block at full
    resolution: each equals full-resolution shading with every 2^i-th sample (a separate
    code path), its AO is a multiple of 1 / ceil(N / 2^i), and no other pixel is written."""
    fr = sg.gbuffer(5, 96, 72, 10, 3)
    N = 48
    cfg = cfg_for("ssao", 4, samples=N, sample_levels=1)
    res = orc.render(fr, cfg)
    for i in (1, 2, 3):
        ci = res["c"][i][..., 0]
        wl = res["lists"][i]
        want = np.zeros(ci.shape, bool)
        for e in wl:
            qy, qx = int(e >> 16), int(e & 0xFFFF)
            want[qy << i:(qy + 1) << i, qx << i:(qx + 1) << i] = True
        assert np.array_equal(np.isfinite(ci), want), i
        thin = orc.level_config(cfg, i)
        assert thin["samples"] == -(-N // (1 << i))
        full = orc.shade_full(fr, dict(thin, sample_levels=0))[..., 0]
        assert np.array_equal(ci[want], full[want]), i
        n_i = thin["samples"]
        occ = (1.0 - ci[want].astype(np.float64)) * n_i
        assert np.allclose(occ, np.round(occ), atol=1e-4), i


def test_sample_levels_merge_gates_on_the_pixels_own_texel():
    """Three levels, the coarsest 0.5; level 1 rendered (c = 1, a = 1, w = 1) on texel
    columns 0..3 only.  Pixel x = 7 (texel 3) reads a_1 = 1 and becomes 1; pixel x = 8 sits
    in texel 4, which was not rendered, so it keeps 0.5 although a_1 interpolates to 1/2
    there.  The direct merge of level-resolution sub-images gives 0.75 at x = 8 (its c_1
    is renormalised over the rendered tap)."""
    H, W = 16, 24
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    w = [0.0, 1.0, 1.0, 0.0]
    cfg_s = cfg_for("ssao", 3, weight=w, enabled=[0, 1, 1, 0], sample_levels=1)
    a = [np.zeros((H, W)), np.zeros((8, 12)), np.ones((4, 6))]
    S = [np.zeros((H, W), np.uint8), np.zeros((8, 12), np.uint8), np.ones((4, 6), np.uint8)]
    a[1][:, :4] = 1.0
    S[1][:, :4] = 1
    full1 = np.full((H, W, 1), np.nan)
    full1[:, :8] = 1.0
    c_s = [np.full((H, W, 1), np.nan), full1, np.full((H, W, 1), 0.5)]
    out = orc.merge(fr, cfg_s, a, S, c_s, "f64")[..., 0]
    assert np.all(out[2:-2, 7] == 1.0) and np.all(out[2:-2, 8] == 0.5)
    c1 = np.full((8, 12, 1), np.nan)
    c1[:, :4] = 1.0
    direct = orc.merge(fr, cfg_for("ssao", 3, weight=w, enabled=[0, 1, 1, 0]), a, S,
                       [np.full((H, W, 1), np.nan), c1, np.full((4, 6, 1), 0.5)], "f64")[..., 0]
    assert np.all(direct[2:-2, 8] == 0.75)


def test_sample_levels_merge_constants_and_eq1():
    H, W = 16, 16
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for("ssao", 2, enabled=[1, 1, 0, 0], weight=[4.0, 1.0, 0, 0], sample_levels=1)
    A, B = 0.25, 0.75
    for a0 in (0.0, 0.05, 0.2, 0.3, 1.0):
        a = [np.full((H, W), a0), np.ones((8, 8))]
        S = [np.ones((H, W), np.uint8), np.ones((8, 8), np.uint8)]
        out = orc.merge(fr, cfg, a, S, [np.full((H, W, 1), A), np.full((H, W, 1), B)], "f64")
        alpha = min(4.0 * a0, 1.0)
        assert np.allclose(out, A * alpha + B * (1 - alpha), rtol=1e-12, atol=1e-12)


def test_sample_levels_with_one_sample_equal_full_resolution():
    """With N = 1 every level keeps the same single sample, so every sub-image equals
    full-resolution shading and the blend returns it (up to the rounding of Eq. (1))."""
    fr = sg.gbuffer(7, 80, 60, 10, 3)
    cfg = cfg_for("ssao", 4, samples=1, sample_levels=1)
    res = orc.render(fr, cfg, "f64")
    full = orc.shade_full(fr, cfg, "f64")
    assert np.allclose(res["out"], full, rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        orc.render(fr, dict(cfg, blur=[0, 1, 1, 1]))


# ----------------------------------------------------------------- pyramid gathers (SSAO)

def test_pyramid_gathers_read_only_the_level_sample_pixels():
    """Depth 2 at the level-2 sample pixels (4q + 2) and 1.5 everywhere else, normals facing
    the camera, radius 0.6.  Level-2 SSAO with pyramid gathers reads only sample pixels, so
    it sees a flat fronto-parallel plane: AO = 1 at every texel.  Reading full resolution,
    the nearer pixels between the samples occlude (0.5 < r)."""
    H, W = 64, 96
    depth = np.full((H, W), 1.5)
    depth[2::4, 2::4] = 2.0
    fr = synthetic_frame(depth, flat_normals(H, W))
    cfg = cfg_for("ssao", 4, samples=32, radius=0.6)
    Hi, Wi = orc.level_dim(H, 2), orc.level_dim(W, 2)
    qy, qx = np.mgrid[0:Hi, 0:Wi]
    wl = ((qy.astype(np.uint32) << 16) | qx.astype(np.uint32)).ravel()
    pyr = orc.shade_level(fr, dict(cfg, pyramid_gathers=1), 2, wl, "f64")[..., 0]
    plain = orc.shade_level(fr, cfg, 2, wl, "f64")[..., 0]
    assert np.all(pyr == 1.0)
    assert plain[2:-2, 2:-2].max() < 1.0


def test_pyramid_gathers_equal_full_resolution_on_block_constant_depth():
    """Depth constant over aligned 8 x 8 blocks: every level-i block (i <= 3) lies inside
    one, so its sample pixel carries the depth of every pixel it stands for and the pyramid
    gathers read exactly what the full-resolution gathers read -- every sub-image equal."""
    rng = np.random.default_rng(4)
    H, W = 48, 72
    blocks = 2.0 + 0.5 * rng.random((H // 8, W // 8))
    depth = np.kron(blocks, np.ones((8, 8)))
    fr = synthetic_frame(depth, flat_normals(H, W))
    cfg = cfg_for("ssao", 4, samples=32, radius=0.6)
    res = orc.render(fr, cfg)
    pyr = orc.render(fr, dict(cfg, pyramid_gathers=1))
    for i in range(4):
        assert np.array_equal(res["lists"][i], pyr["lists"][i])
        assert np.array_equal(res["c"][i], pyr["c"][i], equal_nan=True), i
    assert (res["c"][1][np.isfinite(res["c"][1])] < 1.0).any()   # the steps do occlude


# ----------------------------------------------------------------- sub-image blur (Sec. 4.1)

BINOMIAL = np.array([1.0, 4.0, 6.0, 4.0, 1.0])


def _blur_frame(depth):
    H, W = depth.shape
    return synthetic_frame(depth, flat_normals(H, W))


def test_blur_flat_depth_is_normalised_binomial_convolution():
    """One depth everywhere: the bilateral blur reduces to the normalised convolution
    conv(c S) / conv(S) with the 5x5 binomial kernel (scipy.ndimage), zero outside."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(11)
    H, W, level = 38, 54, 1
    fr = _blur_frame(np.full((H, W), 2.0))
    cfg = cfg_for("ssao", 4)
    Hi, Wi = orc.level_dim(H, level), orc.level_dim(W, level)
    K = np.outer(BINOMIAL, BINOMIAL)
    for density in (1.0, 0.6):
        S = (rng.random((Hi, Wi)) < density).astype(np.uint8)
        c = rng.random((Hi, Wi, 1))
        c[S == 0] = np.nan
        b = orc.blur_level(fr, cfg, level, S, c, "f64")
        cs = np.where(S == 1, c[..., 0], 0.0)
        want = (ndimage.convolve(cs, K, mode="constant", cval=0.0)
                / ndimage.convolve(S.astype(np.float64), K, mode="constant", cval=0.0))
        on = S == 1
        assert np.allclose(b[..., 0][on], want[on], rtol=1e-13, atol=1e-15)
        assert np.all(np.isnan(b[..., 0][~on]))          # unrendered texels are left alone


def test_blur_reproduces_linear_ramps_and_constants():
    """The binomial kernel is symmetric with unit-normalised weights: a constant stays
    exact everywhere and a linear ramp is reproduced two texels from the borders."""
    H, W, level = 40, 48, 2
    fr = _blur_frame(np.full((H, W), 4.0))
    cfg = cfg_for("ssao", 4)
    Hi, Wi = orc.level_dim(H, level), orc.level_dim(W, level)
    S = np.ones((Hi, Wi), np.uint8)
    for prec in ("f32", "f64"):
        b = orc.blur_level(fr, cfg, level, S, np.full((Hi, Wi, 1), 0.625), prec)
        assert np.all(b == 0.625)
    qy, qx = np.mgrid[0:Hi, 0:Wi]
    ramp = (0.125 * qx - 0.0625 * qy + 1.0)[..., None]
    b = orc.blur_level(fr, cfg, level, S, ramp, "f64")
    assert np.array_equal(b[2:-2, 2:-2], ramp[2:-2, 2:-2])


def test_blur_depth_test_is_relative_to_the_centre_texel():
    """Depth 1 left of column k and 0.952 from k on, blur_depth_rel = 0.05: a texel on the
    left takes its right neighbours (|0.048| <= 0.05), one on the right refuses its left
    neighbours (0.048 > 0.0476).  With c = 0 left and 1 right, the texel just left of
    the step reads (B[3] + B[4]) / 16 = 5/16 and every right texel stays 1."""
    level, k = 1, 8
    Hi, Wi = 12, 16
    H, W = 2 * Hi, 2 * Wi
    depth = np.ones((H, W))
    depth[:, 2 * k:] = 0.952
    fr = _blur_frame(depth)
    cfg = cfg_for("ssao", 4, blur_depth_rel=0.05)
    S = np.ones((Hi, Wi), np.uint8)
    c = np.zeros((Hi, Wi, 1))
    c[:, k:] = 1.0
    b = orc.blur_level(fr, cfg, level, S, c, "f64")[..., 0]
    assert np.all(b[:, k:] == 1.0)
    assert np.all(b[2:-2, k - 1] == 5.0 / 16.0)
    assert np.all(b[2:-2, k - 2] == 1.0 / 16.0)
    assert np.all(b[:, : k - 2] == 0.0)
    # a tighter test keeps the two sides apart in both directions
    b = orc.blur_level(fr, cfg_for("ssao", 4, blur_depth_rel=0.04), level, S, c, "f64")[..., 0]
    assert np.all(b[:, :k] == 0.0) and np.all(b[:, k:] == 1.0)


def test_blur_reads_depth_at_the_level_sample_pixels():
    """Level 2 samples pixel 4q + 2.  Depth is 9 at every other pixel; at the sample
    pixels it is 1, and 3 from texel column k on.  Read at the sample pixels, the step
    keeps the two sides apart (c stays 0 | 1); read anywhere else, the depth is flat and
    the texels beside the step would mix to 5/16 and 11/16."""
    level, k = 2, 6
    Hi, Wi = 10, 14
    H, W = 4 * Hi, 4 * Wi
    depth = np.full((H, W), 9.0)
    ys = np.arange(Hi) * 4 + 2
    xs = np.arange(Wi) * 4 + 2
    depth[np.ix_(ys, xs)] = np.where(np.arange(Wi)[None, :] < k, 1.0, 3.0)
    fr = _blur_frame(depth)
    cfg = cfg_for("ssao", 4, blur_depth_rel=0.05)
    c = np.zeros((Hi, Wi, 1))
    c[:, k:] = 1.0
    b = orc.blur_level(fr, cfg, level, np.ones((Hi, Wi), np.uint8), c, "f64")[..., 0]
    assert np.all(b[:, :k] == 0.0) and np.all(b[:, k:] == 1.0)
    flat = orc.blur_level(_blur_frame(np.full((H, W), 9.0)), cfg, level, np.ones((Hi, Wi), np.uint8), c,
                          "f64")[..., 0]
    assert np.all(flat[2:-2, k - 1] == 5.0 / 16.0) and np.all(flat[2:-2, k] == 11.0 / 16.0)


def test_blur_border_window_is_renormalised():
    """At the level's corner only the 3 x 3 quarter of the window lies inside: its
    weights (6 4 1) x (6 4 1) sum to 121, and a unit impulse at the corner reads
    36 / 121 there.  One texel in, a row or column keeps 4 + 6 + 4 + 1 = 15 of its 16."""
    level = 1
    Hi, Wi = 9, 11
    fr = _blur_frame(np.full((2 * Hi, 2 * Wi), 3.0))
    cfg = cfg_for("ssao", 4)
    c = np.zeros((Hi, Wi, 1))
    c[0, 0] = 1.0
    b = orc.blur_level(fr, cfg, level, np.ones((Hi, Wi), np.uint8), c, "f64")[..., 0]
    assert b[0, 0] == 36.0 / 121.0
    # texel (0, 1): rows 0..2 inside (6 + 4 + 1 = 11), columns -1..3 inside (4+6+4+1 = 15)
    assert b[0, 1] == 4.0 * 6.0 / (11.0 * 15.0)
    # texel (1, 1): rows and columns -1..3 inside (15 each); the impulse is at (-1, -1)
    assert b[1, 1] == 16.0 / 225.0


def test_blur_in_render_changes_only_blurred_levels():
    fr = sg.gbuffer(4, 120, 72, 10, 3)
    base = cfg_for("ssao", 4, samples=16)
    res0 = orc.render(fr, base)
    res1 = orc.render(fr, dict(base, blur=[0, 1, 1, 1]))
    assert np.array_equal(res0["c"][0], res1["c"][0], equal_nan=True)
    for i in (1, 2, 3):
        on = res0["S"][i] == 1
        assert not np.array_equal(res0["c"][i][on], res1["c"][i][on])
        assert np.all(np.isfinite(res1["c"][i][on]))
        assert np.all((res1["c"][i][on] >= 0) & (res1["c"][i][on] <= 1))
    assert np.all(np.isfinite(res1["out"]))


# ----------------------------------------------------------------- whole method

def test_cross_level_point_sample_invariant():
    """c_i(q) equals full-resolution shading at s_i(q), bit for bit."""
    fr = sg.gbuffer(1, 130, 77, 10, 3)
    cfg = cfg_for("ssao", 4, samples=16)
    full = orc.shade_full(fr, cfg)
    res = orc.render(fr, cfg)
    for i in range(4):
        wl = res["lists"][i]
        qy, qx = wl >> 16, wl & 0xFFFF
        sy = np.array([orc.level_sample(int(q), i, fr.height) for q in qy])
        sx = np.array([orc.level_sample(int(q), i, fr.width) for q in qx])
        assert np.array_equal(res["c"][i][qy, qx, 0], full[sy, sx, 0])


@pytest.mark.parametrize("effect", ["ssao", "ssgi"])
def test_force_level0_equals_full_resolution_exactly(effect):
    fr = sg.gbuffer(9, 97, 61, 10, 4)
    cfg = cfg_for(effect, 4, samples=16, force_level0=1, radius=0.5 if effect == "ssao" else 1.0)
    res = orc.render(fr, cfg)
    full = orc.shade_full(fr, cfg)
    assert np.all(res["label"] == 0)
    assert np.array_equal(res["out"], full)


def test_multires_error_against_full_resolution_is_small():
    fr = sg.gbuffer(0, 256, 256, 8, 0)
    cfg = cfg_for("ssao", 3, samples=16)
    res = orc.render(fr, cfg)
    full = orc.shade_full(fr, cfg)
    rmse = float(np.sqrt(np.mean((res["out"] - full) ** 2)))
    assert rmse <= 1e-2
    n = sum(len(l) for l in res["lists"])
    assert n < 0.5 * fr.width * fr.height          # far fewer shaded texels than pixels


def test_fp64_and_fp32_oracles_agree_statistically():
    fr = sg.gbuffer(2, 200, 120, 16, 4)
    cfg = cfg_for("ssao", 4, samples=32)
    f32 = orc.render(fr, cfg, "f32")
    f64 = orc.render(fr, cfg, "f64")
    assert np.array_equal(f32["E"], f64["E"]) or np.mean(f32["E"] != f64["E"]) < 1e-3
    diff = f32["out"].astype(np.float64) - f64["out"]
    assert np.sqrt(np.mean(diff ** 2)) < 2e-3
    assert np.quantile(np.abs(diff), 0.999) <= 1.0 / 32 + 1e-6


# ----------------------------------------------------------------- disjoint tiles (Sec. 3.1)

def _single_edge_frame(W=64, H=64, at=(20, 20)):
    """A flat frame whose only edge is one pixel: a depth spike at `at`."""
    d = np.full((H, W), 3.0)
    d[at[1], at[0]] = 2.0
    return synthetic_frame(d, flat_normals(H, W))


@pytest.mark.parametrize("at", [(20, 20), (21, 21), (20, 33)])
def test_disjoint_tiles_two_levels_dead_pixels_closed_form(at):
    """Two levels, one edge pixel: level 0's region is the (2R+1)^2 = 7x7 square around it
    (R = 3); without overlap, level 1 gives up every 2x2 block the square touches, which
    spans 8x8 pixels for a square of odd side wherever it lies, so exactly 8^2 - 7^2 = 15
    pixels belong to no sub-image, and the recomposition leaves exactly those undefined."""
    H = W = 64
    fr = synthetic_frame(np.full((H, W), 3.0), flat_normals(H, W))
    cfg = cfg_for(levels=2, samples=16, disjoint=1)
    E = np.zeros((H, W), np.uint8)
    E[at[1], at[0]] = 1
    a, S, label = orc.masks(fr, cfg, E)
    cov0 = S[0].astype(bool)
    cov1 = np.kron(S[1], np.ones((2, 2), np.uint8))[:H, :W].astype(bool)
    x, y = at
    square = np.zeros((H, W), bool)
    square[y - 3:y + 4, x - 3:x + 4] = True
    assert np.array_equal(cov0, square)
    assert not np.any(cov0 & cov1)                       # disjoint
    dead = ~(cov0 | cov1)
    assert dead.sum() == 15
    hull = np.zeros((H, W), bool)
    hull[(y - 3) // 2 * 2:(y + 3) // 2 * 2 + 2, (x - 3) // 2 * 2:(x + 3) // 2 * 2 + 2] = True
    assert np.array_equal(dead, hull & ~square)
    assert np.all(label[dead] == 255) and np.all(label[cov0] == 0) and np.all(label[cov1] == 1)
    c = [orc.shade_level(fr, cfg, i, orc.compact(S[i])) for i in range(2)]
    out = orc.merge(fr, cfg, a, S, c)[..., 0]
    assert np.array_equal(np.isnan(out), dead)
    assert np.all(out[~dead] == 1.0)                     # a flat plane is unoccluded


@pytest.mark.parametrize("effect", ["ssao", "ssgi"])
def test_disjoint_tiles_are_a_partition_up_to_dead_pixels(effect):
    fr = sg.gbuffer(6, 160, 96, 20, 6)
    cfg = cfg_for(effect, 4, samples=16, disjoint=1)
    E = orc.edges(fr, cfg)
    a, S, label = orc.masks(fr, cfg, E)
    H, W = fr.height, fr.width
    cover = np.zeros((H, W), np.int32)
    for i in range(4):
        if not cfg["enabled"][i]:
            assert S[i].sum() == 0
            continue
        cover += np.kron(S[i].astype(np.int32), np.ones((1 << i, 1 << i), np.int32))[:H, :W]
    assert cover.max() == 1                              # never rendered twice
    assert np.any(cover == 0)                            # dead pixels, as Fig. 4 (left) shows
    out = orc.render(fr, cfg)["out"]
    nan = np.isnan(out[..., 0])
    assert np.all(nan[cover == 0])                       # undefined where no sub-image is
    assert not np.any(nan[(cover == 1) & (label == 0)])  # level 0 is its own pixels


def test_disjoint_tiles_without_dead_pixels_reduce_to_one_level():
    # no edge: only the coarsest level renders, and it covers everything
    H = W = 48
    fr = synthetic_frame(np.full((H, W), 2.5), flat_normals(H, W))
    cfg = cfg_for(samples=16, disjoint=1)
    a, S, label = orc.masks(fr, cfg, orc.edges(fr, cfg))
    assert all(S[i].sum() == 0 for i in range(3)) and S[3].all()
    out = orc.render(fr, cfg)["out"]
    assert not np.isnan(out).any() and np.all(out == 1.0)
    # every pixel at level 0: the full-resolution image exactly
    fr = sg.gbuffer(2, 96, 64, 12, 4)
    cfg = cfg_for(samples=16, disjoint=1, force_level0=1)
    out = orc.render(fr, cfg, "f32")["out"]
    assert np.array_equal(out, orc.shade_full(fr, cfg, "f32"))
