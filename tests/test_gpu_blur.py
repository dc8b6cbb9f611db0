"""The bilateral blur of the rendered sub-images (Sec. 4.1) on the GPU against the
oracle, through the C ABI: the staged mrr_blur_level and the blur inside mrr_render,
the batched path and the serving path's contexts, FP32 and FP16 storage, ragged sizes.

Bars as for the other sub-images: within 1e-4 in FP32 (the kernel takes the oracle's
operations in the oracle's order, so SSAO's blurred sub-images are compared bit for bit
as well), 1e-3 with FP16 storage."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from test_gpu_parity import TOL32, check_frame, make_cfg, run_staged

pytestmark = pytest.mark.gpu

BLUR = [0, 1, 1, 1]


@pytest.fixture(scope="module")
def mrr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


@pytest.mark.parametrize("W,H,seed", [(203, 141, 11), (257, 129, 3), (33, 17, 5), (1, 1, 0), (300, 1, 4)])
def test_ssao_blur_ragged_sizes(mrr, W, H, seed):
    fr = sg.gbuffer(seed, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, blur=BLUR), check_full=False)


def test_ssao_blur_is_bit_exact_fp32(mrr):
    """Same operations, same order: the blurred SSAO sub-images equal the float oracle's
    bit for bit at every listed texel."""
    import torch
    W, H = 240, 150
    fr = sg.gbuffer(7, W, H, 20, 6)
    cfg = make_cfg("ssao", 4, W, H, samples=32, blur=BLUR, blur_depth_rel=0.03)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    _, levels, subs, _ = run_staged(mrr, ctx, dev, W, H, 4)
    for i in (1, 2, 3):
        wl = ref["lists"][i]
        qy, qx = wl >> 16, wl & 0xFFFF
        got = subs[i].cpu().numpy()[qy, qx]
        assert np.array_equal(got.view(np.uint32), ref["c"][i][qy, qx, 0].view(np.uint32)), i
    mrr.mrr_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("effect", ["ssao", "ssgi", "ssm"])
def test_blur_every_effect_and_storage(mrr, effect, precision):
    W, H = 170, 100
    fr = sg.gbuffer(8, W, H, 20, 6, shadow_size=512 if effect == "ssm" else 0)
    blur = [0, 0, 1, 1] if effect == "ssgi" else BLUR     # SSGI has no level 1
    cfg = make_cfg(effect, 4, W, H, precision, blur=blur)
    check_frame(mrr, fr, cfg, precision, check_full=False)


def test_blur_sky_and_depth_steps(mrr):
    """A frame with sky above the horizon: sky texels of the coarse levels and surface
    texels never mix (their depths differ by far more than the test allows)."""
    W, H = 128, 96
    fr = sg.gbuffer(2, W, H, 12, 4, eye=(0.0, 1.0, 6.0), target=(0.0, 1.2, 0.0))
    assert np.any(fr.depth >= fr.cam.far) and np.any(fr.depth < fr.cam.far)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, blur=BLUR), check_full=False)


def test_blur_arguments_are_validated(mrr):
    import torch
    W, H = 64, 48
    fr = sg.gbuffer(0, W, H, 6, 2)
    for bad in ([1, 0, 0, 0], [0, 2, 0, 0]):
        with pytest.raises(mrr.MrrError) as ei:
            mrr.mrr_create(make_cfg("ssao", 4, W, H, blur=bad))
        assert ei.value.status == mrr.MRR_EINVAL
    with pytest.raises(mrr.MrrError):                       # level beyond num_levels
        mrr.mrr_create(make_cfg("ssao", 3, W, H, blur=[0, 0, 0, 1]))
    with pytest.raises(mrr.MrrError):                       # SSGI's disabled level 1
        mrr.mrr_create(make_cfg("ssgi", 4, W, H, blur=[0, 1, 0, 0]))
    with pytest.raises(mrr.MrrError):
        mrr.mrr_create(make_cfg("ssao", 4, W, H, blur=BLUR, blur_depth_rel=-0.1))
    ctx = mrr.mrr_create(make_cfg("ssao", 4, W, H))
    dev = mrr.upload_frame(fr)
    _, levels, subs, _ = run_staged(mrr, ctx, dev, W, H, 4)
    before = mrr.mrr_kernel_launches()
    for level, c, b in ((0, subs[0], torch.empty_like(subs[0])), (1, subs[1], subs[1]), (4, subs[1], subs[2])):
        with pytest.raises(mrr.MrrError) as ei:
            mrr.mrr_blur_level(ctx, level, dev, levels, c, b)
        assert ei.value.status == mrr.MRR_EINVAL
    assert mrr.mrr_kernel_launches() == before              # nothing was launched
    mrr.mrr_destroy(ctx)


def test_blur_in_batches_equals_single_frames(mrr):
    import torch
    ctxs, frames, outs, refs = [], [], [], []
    for effect, W, H, prec, seed in [("ssao", 200, 120, "fp32", 1), ("ssgi", 160, 96, "fp16", 2),
                                     ("ssao", 131, 77, "fp16", 3)]:
        fr = sg.gbuffer(seed, W, H, 16, 4)
        cfg = make_cfg(effect, 4, W, H, prec, blur=[0, 0, 1, 1] if effect == "ssgi" else BLUR)
        ctx = mrr.mrr_create(cfg)
        dev = mrr.upload_frame(fr, prec)
        ref = mrr.alloc_output(ctx, W, H)
        mrr.mrr_render(ctx, dev, ref)
        ctxs.append(ctx)
        frames.append(dev)
        outs.append(mrr.alloc_output(ctx, W, H))
        refs.append(ref)
    b = mrr.mrr_batch_create()
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        mrr.mrr_render_batch(b, ctxs, frames, outs)
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
    mrr.mrr_batch_destroy(b)
    for c in ctxs:
        mrr.mrr_destroy(c)


def test_ssao64_1080p_blurred_full_size(mrr):
    """The 1920x1080 SSAO-64 workload with levels 1-3 blurred, in the launch configuration
    the benchmark times: the composite against the oracle over the whole frame, and the
    blurred image's RMSE against unblurred full-resolution shading."""
    import torch
    wl = sg.WORKLOADS["ssao64_1080p"]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"])
    cfg = make_cfg("ssao", 4, W, H, samples=64, blur=BLUR)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out, full = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    mrr.mrr_render_full(ctx, dev, full)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.abs(o - ref["out"][..., 0]).max() <= TOL32
    assert mrr.mrr_fault_flags(ctx) == 0
    assert float(np.sqrt(np.mean((o - full.cpu().numpy()) ** 2))) <= 1e-2
    mrr.mrr_destroy(ctx)
