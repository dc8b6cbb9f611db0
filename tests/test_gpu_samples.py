"""Sample-count levels (Sec. 6; mrr_config.sample_levels = 1) on the GPU against the
oracle, through the C ABI: levels above 0 rendered at full resolution over their
texels' blocks with every 2^i-th sample, blended without upsampling.  Staged calls
(mrr_shade_level / mrr_shade_levels / mrr_upsample_merge), mrr_render, batches; every
effect and storage precision; ragged sizes.

Bars: masks and lists bit-exact (unchanged stages); sub-images and composite within
1e-4 in FP32 (the same operations in the same order), 1e-3 with FP16 storage;
mrr_render equals the staged path bit for bit."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from test_gpu_parity import TOL16, TOL32, make_cfg, oracle_inputs

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


def check_samples(mrr, fr, cfg, precision="fp32", one_call=True):
    import torch
    W, H, L = fr.width, fr.height, cfg["num_levels"]
    C = 3 if cfg["effect"] == "ssgi" else 1
    tol = TOL16 if precision == "fp16" else TOL32
    ref = orc.render(oracle_inputs(fr, precision), cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr, precision)
    edges = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    levels = mrr.alloc_levels(W, H, L)
    subs = mrr.alloc_subimages(ctx, W, H)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_edges(ctx, dev, edges)
    mrr.mrr_masks(ctx, edges, levels)
    if one_call:
        mrr.mrr_shade_levels(ctx, dev, levels, subs)
    else:
        for i in range(L):
            if cfg["enabled"][i]:
                mrr.mrr_shade_level(ctx, i, dev, levels, subs[i])
    mrr.mrr_upsample_merge(ctx, levels, subs, out)
    torch.cuda.synchronize()
    for i in range(L):
        assert np.array_equal(levels.stencil[i].cpu().numpy(), ref["S"][i]), i
        if not cfg["enabled"][i]:
            continue
        got = subs[i].float().cpu().numpy()
        got = got if C == 1 else got[..., :3]
        exp = ref["c"][i][..., 0] if C == 1 else ref["c"][i]
        on = np.isfinite(exp) if C == 1 else np.isfinite(exp[..., 0])
        assert np.array_equal(np.isfinite(got if C == 1 else got[..., 0]), on), f"written pixels of level {i}"
        assert np.abs(got[on] - exp[on]).max(initial=0.0) <= tol, f"sub-image {i}"
    o = out.cpu().numpy()
    o = o if C == 1 else o[..., :3]
    e = ref["out"][..., 0] if C == 1 else ref["out"]
    assert np.abs(o - e).max() <= tol, f"composite {np.abs(o - e).max()}"
    out2 = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out2)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    mrr.mrr_destroy(ctx)


@pytest.mark.parametrize("W,H,seed", [(203, 141, 11), (33, 17, 5), (1, 1, 0), (7, 3, 2), (300, 1, 4)])
def test_sample_levels_ragged_sizes(mrr, W, H, seed):
    fr = sg.gbuffer(seed, W, H, 16, 6)
    check_samples(mrr, fr, make_cfg("ssao", 4, W, H, samples=24, sample_levels=1))


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("effect", ["ssao", "ssgi", "ssm"])
def test_sample_levels_every_effect_and_storage(mrr, effect, precision):
    W, H = 150, 96
    fr = sg.gbuffer(8, W, H, 20, 6, shadow_size=512 if effect == "ssm" else 0)
    check_samples(mrr, fr, make_cfg(effect, 4, W, H, precision, sample_levels=1), precision,
                  one_call=effect != "ssm")


def test_sample_levels_config_is_validated(mrr):
    for kw in (dict(blur=[0, 1, 1, 1]), dict(merge_mode=1), dict(sample_levels=3)):
        with pytest.raises(mrr.MrrError) as ei:
            mrr.mrr_create(make_cfg("ssao", 4, 64, 48, sample_levels=kw.pop("sample_levels", 1), **kw))
        assert ei.value.status == mrr.MRR_EINVAL


def test_sample_levels_in_batches_equal_single_frames(mrr):
    import torch
    ctxs, frames, outs, refs = [], [], [], []
    for effect, W, H, prec, seed, sl in [("ssao", 200, 120, "fp32", 1, 1), ("ssgi", 160, 96, "fp16", 2, 1),
                                         ("ssao", 131, 77, "fp32", 3, 0)]:
        fr = sg.gbuffer(seed, W, H, 16, 4)
        cfg = make_cfg(effect, 4, W, H, prec, sample_levels=sl)
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


def test_ssao64_1080p_sample_levels_full_size(mrr):
    """The 1920x1080 SSAO-64 workload with sample-count levels, in the launch
    configuration the benchmark times: the composite against the oracle over the whole
    frame."""
    import torch
    wl = sg.WORKLOADS["ssao64_1080p"]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"])
    cfg = make_cfg("ssao", 4, W, H, samples=64, sample_levels=1)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref["out"][..., 0]).max() <= TOL32
    assert mrr.mrr_fault_flags(ctx) == 0
    mrr.mrr_destroy(ctx)
