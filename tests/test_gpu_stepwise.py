"""The step-wise blending of Sec. 3.3 (merge_mode 1) on the GPU against the oracle,
through the C ABI: the staged mrr_upsample_merge and mrr_render (whose level 0 is
blended over its list), batches, every effect and storage precision, ragged sizes,
two to four levels, and the skipped 1/2 level of SSGI (a 4x step).

Bars as for the direct merge: within 1e-4 in FP32 (same operations in the same order,
so equality is expected), 1e-3 with FP16 storage; mrr_render equals the staged path bit
for bit."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from test_gpu_parity import TOL32, check_frame, make_cfg

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


@pytest.mark.parametrize("W,H,seed", [(203, 141, 11), (257, 129, 3), (33, 17, 5), (1, 1, 0), (7, 3, 2), (300, 1, 4)])
def test_stepwise_ragged_sizes(mrr, W, H, seed):
    fr = sg.gbuffer(seed, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, merge_mode=1), check_full=False)


@pytest.mark.parametrize("levels", [2, 3])
def test_stepwise_fewer_levels(mrr, levels):
    W, H = 150, 90
    fr = sg.gbuffer(6, W, H, 12, 4)
    check_frame(mrr, fr, make_cfg("ssao", levels, W, H, samples=16, merge_mode=1), check_full=False)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("effect", ["ssao", "ssgi", "ssm"])
def test_stepwise_every_effect_and_storage(mrr, effect, precision):
    W, H = 170, 100
    fr = sg.gbuffer(8, W, H, 20, 6, shadow_size=512 if effect == "ssm" else 0)
    cfg = make_cfg(effect, 4, W, H, precision, merge_mode=1)
    check_frame(mrr, fr, cfg, precision, check_full=False)


def test_stepwise_with_blur(mrr):
    W, H = 190, 110
    fr = sg.gbuffer(9, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=16, merge_mode=1, blur=[0, 1, 1, 1]),
                check_full=False)


def test_stepwise_staged_merge_needs_pool_size(mrr):
    import torch
    W, H = 64, 48
    fr = sg.gbuffer(0, W, H, 6, 2)
    ctx = mrr.mrr_create(make_cfg("ssao", 4, 32, 32, merge_mode=1))
    levels = mrr.alloc_levels(W, H, 4)
    subs = [torch.zeros((orc.level_dim(H, i), orc.level_dim(W, i)), device="cuda") for i in range(4)]
    out = torch.empty((H, W), device="cuda")
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_upsample_merge(ctx, levels, subs, out)
    assert ei.value.status == mrr.MRR_EINVAL
    mrr.mrr_destroy(ctx)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_create(make_cfg("ssao", 4, W, H, merge_mode=3))


def test_stepwise_in_batches_equals_single_frames(mrr):
    import torch
    ctxs, frames, outs, refs = [], [], [], []
    for effect, W, H, prec, seed in [("ssao", 200, 120, "fp32", 1), ("ssgi", 160, 96, "fp16", 2),
                                     ("ssm", 131, 77, "fp32", 3)]:
        fr = sg.gbuffer(seed, W, H, 16, 4, shadow_size=512 if effect == "ssm" else 0)
        cfg = make_cfg(effect, 4, W, H, prec, merge_mode=1)
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


def test_ssao64_1080p_stepwise_full_size(mrr):
    """The 1920x1080 SSAO-64 workload with step-wise blending, in the launch configuration
    the benchmark times: the composite against the oracle over the whole frame and its
    RMSE against full-resolution shading."""
    import torch
    wl = sg.WORKLOADS["ssao64_1080p"]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"])
    cfg = make_cfg("ssao", 4, W, H, samples=64, merge_mode=1)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out, full = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    mrr.mrr_render_full(ctx, dev, full)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.abs(o - ref["out"][..., 0]).max() <= TOL32
    assert float(np.sqrt(np.mean((o - full.cpu().numpy()) ** 2))) <= 1e-2
    mrr.mrr_destroy(ctx)
