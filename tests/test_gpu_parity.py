"""GPU parity: every stage of the CUDA path against the CPU oracle on the same seeded
inputs, through the C ABI.

Bars: edge maps, stencils, blurred masks a_i, work lists, counts and labels
bit-exact (the kernels make every decision in FP32 with the oracle's operation
order); sub-images and composites within 1e-4 absolute in FP32 (bit-equality is
expected); the FP16-storage path against the float oracle fed the same
binary16-rounded inputs, within 1e-3 (one binary16 ulp at 1.0 is 9.8e-4).
"""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL16 = 1e-3


@pytest.fixture(scope="module")
def mrr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


def oracle_inputs(fr, precision):
    """The oracle sees exactly what the kernels read: binary16-rounded colour always,
    binary16-rounded normals in FP16 storage (the shadow map's light depth, like the view
    depth, stays FP32 in both precisions)."""
    import copy
    o = copy.copy(fr)
    o.color = fr.color.astype(np.float16).astype(np.float32)
    if precision == "fp16":
        o.normal = fr.normal.astype(np.float16).astype(np.float32)
    return o


def make_cfg(effect, levels, W, H, precision="fp32", **kw):
    extra = {}
    if effect in ("ssao", "ssgi"):
        n = kw.pop("samples", 16)
        extra.update(samples=n, kernel=sg.hemisphere_kernel(n), radius=kw.pop("radius", 0.5 if effect == "ssao" else 1.0))
    else:
        extra.update(blocker_taps=sg.disk_taps(kw.pop("nb", 32), sg.BLOCKER_SEED),
                     pcf_taps=sg.disk_taps(kw.pop("np_", 64), sg.PCF_SEED))
    extra.update(kw)
    cfg = orc.default_config(effect, levels, store_half=int(precision == "fp16"), **extra)
    cfg.update(precision=precision, max_width=W, max_height=H)
    return cfg


def run_staged(mrr, ctx, dev, W, H, L):
    import torch
    edges = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    levels = mrr.alloc_levels(W, H, L)
    subs = mrr.alloc_subimages(ctx, W, H)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_edges(ctx, dev, edges)
    mrr.mrr_masks(ctx, edges, levels)
    for i in range(L):
        if ctx.config["enabled"][i]:
            mrr.mrr_shade_level(ctx, i, dev, levels, subs[i])
    blur = ctx.config.get("blur", [0, 0, 0, 0])
    for i in range(L):
        if blur[i]:                       # Sec. 4.1 blur into a fresh sub-image
            b = torch.full_like(subs[i], float("nan"))
            mrr.mrr_blur_level(ctx, i, dev, levels, subs[i], b)
            subs[i] = b
    if ctx.config.get("merge_mode", 0) == 2:      # the bilateral merge reads the frame's depth
        mrr.mrr_upsample_merge_bilateral(ctx, dev, levels, subs, out)
    else:
        mrr.mrr_upsample_merge(ctx, levels, subs, out)
    torch.cuda.synchronize()
    return edges, levels, subs, out


def check_frame(mrr, fr, cfg, precision="fp32", check_full=True):
    import torch
    W, H, L = fr.width, fr.height, cfg["num_levels"]
    ofr = oracle_inputs(fr, precision)
    ref = orc.render(ofr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr, precision)
    edges, levels, subs, out = run_staged(mrr, ctx, dev, W, H, L)
    tol = TOL16 if precision == "fp16" else TOL32
    C = 3 if cfg["effect"] == "ssgi" else 1

    assert np.array_equal(edges.cpu().numpy(), ref["E"]), "edge map"
    counts = levels.counts.cpu().numpy()
    for i in range(L):
        assert np.array_equal(levels.stencil[i].cpu().numpy(), ref["S"][i]), f"stencil {i}"
        assert np.array_equal(levels.alpha[i].cpu().numpy().view(np.uint32),
                              ref["a"][i].view(np.uint32)), f"alpha {i} (bit pattern)"
        n = len(ref["lists"][i])
        assert counts[i] == n, f"count {i}"
        if n:
            assert np.array_equal(levels.worklist[i][:n].cpu().numpy().view(np.uint32), ref["lists"][i]), f"list {i}"
            wl = ref["lists"][i]
            qy, qx = wl >> 16, wl & 0xFFFF
            got = subs[i].float().cpu().numpy()
            got = got[qy, qx] if C == 1 else got[qy, qx, :3]
            exp = ref["c"][i][qy, qx, 0] if C == 1 else ref["c"][i][qy, qx, :]
            assert np.abs(got - exp).max() <= tol, f"sub-image {i}: {np.abs(got - exp).max()}"
    assert np.array_equal(levels.label.cpu().numpy(), ref["label"]), "label"
    got = out.cpu().numpy()
    got = got if C == 1 else got[..., :3]
    exp = ref["out"][..., 0] if C == 1 else ref["out"]
    assert np.abs(got - exp).max() <= tol, f"composite: {np.abs(got - exp).max()}"

    # the one-call path equals the staged path bit for bit
    out2 = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out2)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    assert mrr.mrr_fault_flags(ctx) == 0
    if check_full:
        full = mrr.alloc_output(ctx, W, H)
        mrr.mrr_render_full(ctx, dev, full)
        torch.cuda.synchronize()
        exp_full = orc.shade_full(ofr, cfg, "f32")
        g = full.cpu().numpy()
        g = g if C == 1 else g[..., :3]
        e = exp_full[..., 0] if C == 1 else exp_full
        assert np.abs(g - e).max() <= TOL32, f"full-res: {np.abs(g - e).max()}"
    mrr.mrr_destroy(ctx)
    return ref


# ------------------------------------------------------------------ SSAO

def test_ssao_256_three_levels(mrr):
    fr = sg.gbuffer(0, 256, 256, 8, 0)
    check_frame(mrr, fr, make_cfg("ssao", 3, 256, 256, samples=16))


@pytest.mark.parametrize("W,H,seed", [(203, 141, 11), (257, 129, 3), (33, 17, 5), (1, 1, 0), (7, 3, 2), (300, 1, 4)])
def test_ssao_ragged_sizes(mrr, W, H, seed):
    fr = sg.gbuffer(seed, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=64))


@pytest.mark.parametrize("W,H", [(16384, 40), (40, 16384), (16383, 9)])
def test_maximum_dimension_frames(mrr, W, H):
    """Frames at the largest supported width or height (16384): work-list coordinates use
    all 14 bits of their 16-bit fields, the TMA edge kernel walks 512 tiles along a row,
    and a width one below the limit takes the edge kernel without TMA."""
    fr = sg.gbuffer(W % 97 + H, W, H, 24, 8)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16), check_full=False)


def test_dimension_limit_is_enforced(mrr):
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_create(make_cfg("ssao", 4, 16385, 8))
    assert ei.value.status == mrr.MRR_EINVAL


@pytest.mark.parametrize("sigma2", [[0.5, 1.0, 2.5, 0.0], [0.3, 0.924, 3.696, 0.0], [1.848, 3.696, 0.924, 0.0]])
def test_masks_other_radii(mrr, sigma2):
    """Radii other than Table 1's (3, 5, 6) take the mask kernel that carries every radius;
    Table 1's patterns take kernels compiled for them.  Both match the oracle bit for bit."""
    W, H = 203, 141
    fr = sg.gbuffer(12, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, sigma2=sigma2), check_full=False)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("W,H", [(100, 37), (36, 18), (4, 1), (1924, 33), (64, 300)])
def test_edges_tile_staged_sizes(mrr, W, H, precision):
    """Rows a multiple of 16 bytes take the TMA-staged edge kernel: partial 32x16 tiles,
    one-pixel frames and halos outside the image all match the oracle bit for bit."""
    import torch
    fr = sg.gbuffer(W + H, W, H, 24, 8)
    cfg = make_cfg("ssao", 4, W, H, precision)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr, precision)
    edges = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    mrr.mrr_edges(ctx, dev, edges)
    ref = orc.edges(oracle_inputs(fr, precision), cfg, "f32")
    assert np.array_equal(edges.cpu().numpy(), ref)
    assert mrr.mrr_fault_flags(ctx) == 0
    mrr.mrr_destroy(ctx)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ssao_fp16_storage(mrr, seed):
    fr = sg.gbuffer(seed, 190, 110, 20, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, 190, 110, "fp16", samples=32), "fp16")


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_ssao_64_sample_variant(mrr, precision):
    """64 samples with one lane per texel run the kernels compiled for that count (the
    unrolled sample loop); the work lists, the full-resolution image and the frame must
    match the oracle exactly as the runtime-count kernels do."""
    W, H = 173, 101
    fr = sg.gbuffer(7, W, H, 20, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, precision, samples=64, lanes_per_texel=1, lanes_per_pixel=1),
                precision)


def test_all_sky_frame(mrr):
    W, H = 64, 40
    fr = sg.gbuffer(0, W, H, 0, 0, eye=(0.0, 2.0, 6.0), target=(0.0, 20.0, 0.0))   # looking up: sky only
    assert np.all(fr.depth >= fr.cam.far)
    ref = check_frame(mrr, fr, make_cfg("ssao", 4, W, H))
    assert ref["E"].sum() == 0 and np.all(ref["out"] == 1.0)


def test_dense_edges_everywhere(mrr):
    """Noise depth: every pixel is an edge, so level 0 covers the whole frame."""
    W, H = 96, 64
    fr = sg.gbuffer(0, W, H, 0, 0)
    rng = np.random.default_rng(0)
    fr.depth = (2.0 + rng.random((H, W))).astype(np.float32)
    fr.normal[:] = np.array([0, 0, 1, 0], np.float32)
    ref = check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16))
    assert np.all(ref["label"] == 0)


def test_force_level0_equals_full_resolution_on_gpu(mrr):
    import torch
    W, H = 160, 90
    fr = sg.gbuffer(6, W, H, 12, 4)
    cfg = make_cfg("ssao", 4, W, H, samples=32, force_level0=1)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out, full = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    mrr.mrr_render_full(ctx, dev, full)
    torch.cuda.synchronize()
    assert torch.equal(out, full)
    assert np.array_equal(full.cpu().numpy(), orc.shade_full(fr, cfg, "f32")[..., 0])


# ------------------------------------------------------------------ SSGI / SSM

@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_ssgi_skips_half_level(mrr, precision):
    W, H = 170, 100
    fr = sg.gbuffer(8, W, H, 20, 6)
    cfg = make_cfg("ssgi", 4, W, H, precision, samples=32, radius=1.0)
    assert cfg["enabled"] == [1, 0, 1, 1]
    ref = check_frame(mrr, fr, cfg, precision)
    assert len(ref["lists"][1]) == 0


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("size", [(180, 120), (196, 75), (170, 64)])
def test_ssm_soft_shadows(mrr, precision, size):
    """Soft shadows: rows a multiple of 16 bytes take the two-pass edge path (hard-shadow
    bits, then the TMA kernel; 196 x 75 has a partial last bit word and a ragged last tile
    row), other widths the one-pass staged kernel (170)."""
    W, H = size
    fr = sg.gbuffer(4, W, H, 16, 4, shadow_size=512)
    check_frame(mrr, fr, make_cfg("ssm", 4, W, H, precision), precision)


# ------------------------------------------------------------------ full-size workload samples

def test_ssao64_1080p_full_size(mrr):
    """The 1920x1080 SSAO-64 workload in the launch configuration the benchmark times:
    masks and lists bit-exact over the whole frame; the composite against the oracle
    over the whole frame."""
    import torch
    wl = sg.WORKLOADS["ssao64_1080p"]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"])
    cfg = make_cfg("ssao", 4, W, H, samples=64)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref["out"][..., 0]).max() <= TOL32
    edges, levels, subs, out2 = run_staged(mrr, ctx, dev, W, H, 4)
    assert np.array_equal(edges.cpu().numpy(), ref["E"])
    for i in range(4):
        assert np.array_equal(levels.stencil[i].cpu().numpy(), ref["S"][i])
        n = len(ref["lists"][i])
        assert levels.counts[i].item() == n
        assert np.array_equal(levels.worklist[i][:n].cpu().numpy().view(np.uint32), ref["lists"][i])
    # sampled full-resolution pixels of the plain kernel against the oracle one by one
    full = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render_full(ctx, dev, full)
    torch.cuda.synchronize()
    g = full.cpu().numpy()
    rng = np.random.default_rng(0)
    for _ in range(400):
        x, y = int(rng.integers(W)), int(rng.integers(H))
        assert abs(g[y, x] - orc.shade_pixel(fr, cfg, x, y, "f32")[0]) <= TOL32
    # the quality gate of the method: RMSE against full-resolution shading
    assert float(np.sqrt(np.mean((out.cpu().numpy() - g) ** 2))) <= 1e-2
    mrr.mrr_destroy(ctx)


def test_render_host_matches_device_path(mrr):
    import torch
    W, H = 200, 120
    fr = sg.gbuffer(2, W, H, 16, 4)
    cfg = make_cfg("ssao", 4, W, H, samples=32)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    host = mrr.pin_frame(fr)
    out_h = torch.empty((H, W), dtype=torch.float32).pin_memory()
    mrr.mrr_render_host(ctx, host, out_h)
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), out_h)
    mrr.mrr_destroy(ctx)


@pytest.mark.parametrize("effect", ["ssao", "ssgi", "ssm"])
def test_pipelined_host_rendering_matches_device_path(mrr, effect):
    """Five different frames through mrr_render_host_async (two device sets in turn, copies
    overlapping rendering), then one wait: every image equals mrr_render of the same frame
    on the device, bit for bit."""
    import torch
    W, H = 176, 100
    cfg = make_cfg(effect, 4, W, H, samples=16)
    ctx = mrr.mrr_create(cfg)
    frames = [sg.gbuffer(s, W, H, 12, 4, shadow_size=256 if effect == "ssm" else 0) for s in range(5)]
    refs = []
    for fr in frames:
        dev = mrr.upload_frame(fr)
        out = mrr.alloc_output(ctx, W, H)
        mrr.mrr_render(ctx, dev, out)
        torch.cuda.synchronize()
        refs.append(out.cpu())
    hosts = [mrr.pin_frame(fr) for fr in frames]
    outs = [torch.full(tuple(refs[0].shape), float("nan")).pin_memory() for _ in frames]
    for h, o in zip(hosts, outs):
        mrr.mrr_render_host_async(ctx, h, o)
    mrr.mrr_render_host_wait(ctx)
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    mrr.mrr_destroy(ctx)


def test_graph_replay_matches_direct_launches(mrr):
    import torch
    W, H = 220, 130
    frames = [sg.gbuffer(s, W, H, 16, 4) for s in (1, 2)]
    outs = {}
    for no_graph in (0, 1):
        cfg = make_cfg("ssao", 4, W, H, samples=32, no_graph=no_graph)
        ctx = mrr.mrr_create(cfg)
        res = []
        for fr in frames + frames:      # new descriptor, new descriptor, then repeats
            dev = mrr.upload_frame(fr)
            out = mrr.alloc_output(ctx, W, H)
            for _ in range(2):
                mrr.mrr_render(ctx, dev, out)
            torch.cuda.synchronize()
            res.append(out.clone())
        outs[no_graph] = res
        mrr.mrr_destroy(ctx)
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    assert torch.equal(outs[0][0], outs[0][2]) and not torch.equal(outs[0][0], outs[0][1])


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_lane_split_does_not_change_results(mrr, lanes):
    import torch
    W, H = 150, 90
    fr = sg.gbuffer(3, W, H, 12, 4)
    cfg = make_cfg("ssao", 4, W, H, samples=64, lanes_per_texel=lanes, lanes_per_pixel=lanes)
    ref = orc.render(fr, cfg, "f32")
    full_ref = orc.shade_full(fr, cfg, "f32")[..., 0]
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out, full = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    mrr.mrr_render_full(ctx, dev, full)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref["out"][..., 0]).max() <= TOL32
    assert np.array_equal(full.cpu().numpy(), full_ref)
    mrr.mrr_destroy(ctx)


@pytest.mark.parametrize("effect", ["ssao", "ssgi"])
def test_autotune_keeps_results(mrr, effect):
    import torch
    W, H = 240, 136
    fr = sg.gbuffer(5, W, H, 16, 4)
    cfg = make_cfg(effect, 4, W, H, samples=32)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    before, after = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, before)
    t = mrr.mrr_autotune(ctx, dev)
    assert t["lanes_per_texel"] in (1, 2, 4) and t["grid_multiplier"] in (1, 2, 4)
    assert t["shade_levels_ms"] > 0 and t["shade_full_ms"] > 0 and t["candidates"] >= 4
    mrr.mrr_render(ctx, dev, after)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    mrr.mrr_destroy(ctx)


def test_frame_larger_than_context_is_rejected(mrr):
    W, H = 64, 64
    fr = sg.gbuffer(0, W, H, 4, 0)
    cfg = make_cfg("ssao", 4, 32, 32)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out = mrr.alloc_output(ctx, W, H)
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_render(ctx, dev, out)
    assert ei.value.status == mrr.MRR_EINVAL
    mrr.mrr_destroy(ctx)


def test_trace_shading_hook(mrr):
    """mrr_trace_shading: events around the frame path's shading launch give a positive
    device time; the traced (graph-less) render equals the graph replay bit for bit."""
    import torch
    W, H = 160, 96
    fr = sg.gbuffer(2, W, H, 16, 4)
    cfg = make_cfg("ssao", 4, W, H, samples=64)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    ref, got = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, ref)
    tb, te = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mrr.mrr_trace_shading(ctx, tb, te)
    mrr.mrr_render(ctx, dev, got)
    torch.cuda.synchronize()
    assert tb.elapsed_time(te) > 0.0
    mrr.mrr_trace_shading(ctx)
    assert torch.equal(ref, got)
    with pytest.raises(ValueError):
        mrr.mrr_trace_shading(ctx, tb, None)
    mrr.mrr_destroy(ctx)
