"""The direct merge with bilateral (depth-aware) taps (Sec. 3.3; merge_mode 2) on the GPU
against the oracle, through the C ABI: mrr_upsample_merge_bilateral and mrr_render,
batches, every effect and storage precision, ragged sizes, with and without the blur.
Bars as for the other merges: 1e-4 in FP32, 1e-3 with FP16 storage, mrr_render equal to
the staged calls bit for bit."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from test_gpu_parity import TOL32, check_frame, make_cfg, run_staged

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


@pytest.mark.parametrize("W,H,seed", [(203, 141, 11), (33, 17, 5), (1, 1, 0), (300, 1, 4)])
def test_bilateral_ragged_sizes(mrr, W, H, seed):
    fr = sg.gbuffer(seed, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, merge_mode=2), check_full=False)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("effect", ["ssao", "ssgi", "ssm"])
def test_bilateral_every_effect_and_storage(mrr, effect, precision):
    W, H = 170, 100
    fr = sg.gbuffer(8, W, H, 20, 6, shadow_size=512 if effect == "ssm" else 0)
    check_frame(mrr, fr, make_cfg(effect, 4, W, H, precision, merge_mode=2), precision, check_full=False)


def test_bilateral_with_blur_and_three_levels(mrr):
    W, H = 190, 110
    fr = sg.gbuffer(9, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, merge_mode=2, blur=[0, 1, 1, 1]), check_full=False)
    check_frame(mrr, fr, make_cfg("ssao", 3, W, H, samples=16, merge_mode=2), check_full=False)


def test_plain_merge_call_is_refused(mrr):
    import torch
    W, H = 64, 48
    fr = sg.gbuffer(0, W, H, 6, 2)
    ctx = mrr.mrr_create(make_cfg("ssao", 4, W, H, merge_mode=2))
    dev = mrr.upload_frame(fr)
    _, levels, subs, _ = run_staged(mrr, ctx, dev, W, H, 4)
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_upsample_merge(ctx, levels, subs, torch.empty((H, W), device="cuda"))
    assert ei.value.status == mrr.MRR_EINVAL
    mrr.mrr_destroy(ctx)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_create(make_cfg("ssao", 4, W, H, merge_mode=3))


def test_bilateral_in_batches_equals_single_frames(mrr):
    import torch
    ctxs, frames, outs, refs = [], [], [], []
    for effect, W, H, prec, seed in [("ssao", 200, 120, "fp32", 1), ("ssgi", 160, 96, "fp16", 2),
                                     ("ssm", 131, 77, "fp32", 3)]:
        fr = sg.gbuffer(seed, W, H, 16, 4, shadow_size=512 if effect == "ssm" else 0)
        ctx = mrr.mrr_create(make_cfg(effect, 4, W, H, prec, merge_mode=2))
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


def test_ssao64_1080p_bilateral_full_size(mrr):
    import torch
    wl = sg.WORKLOADS["ssao64_1080p"]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"])
    cfg = make_cfg("ssao", 4, W, H, samples=64, merge_mode=2)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref["out"][..., 0]).max() <= TOL32
    mrr.mrr_destroy(ctx)
