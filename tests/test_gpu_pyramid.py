"""Pyramid gathers (SSAO; mrr_config.pyramid_gathers = 1) on the GPU against the oracle,
through the C ABI: the levels above 0 read their depth gathers from the level's point
samples.  Staged calls and mrr_render, FP32 and FP16 storage, ragged sizes, three and
four levels; batches and servers refuse the option.  Bars as elsewhere: 1e-4 in FP32,
1e-3 with FP16 storage, mrr_render equal to the staged calls bit for bit."""
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


@pytest.mark.parametrize("W,H,seed", [(203, 141, 11), (257, 129, 3), (33, 17, 5), (1, 1, 0), (300, 1, 4)])
def test_pyramid_ragged_sizes(mrr, W, H, seed):
    fr = sg.gbuffer(seed, W, H, 16, 6)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=24, pyramid_gathers=1), check_full=False)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("levels", [3, 4])
def test_pyramid_storage_and_levels(mrr, precision, levels):
    W, H = 180, 110
    fr = sg.gbuffer(7, W, H, 20, 6)
    check_frame(mrr, fr, make_cfg("ssao", levels, W, H, precision, samples=32, pyramid_gathers=1), precision,
                check_full=False)


@pytest.mark.parametrize("split", [1, 2, 4])
def test_pyramid_lane_split_keeps_results(mrr, split):
    W, H = 150, 90
    fr = sg.gbuffer(3, W, H, 12, 4)
    check_frame(mrr, fr, make_cfg("ssao", 4, W, H, samples=64, pyramid_gathers=1, lanes_per_texel=split),
                check_full=False)


def test_pyramid_is_refused_where_it_does_not_apply(mrr):
    W, H = 64, 48
    for kw in (dict(effect="ssgi"), dict(effect="ssm"), dict(effect="ssao", sample_levels=1)):
        eff = kw.pop("effect")
        with pytest.raises(mrr.MrrError) as ei:
            mrr.mrr_create(make_cfg(eff, 4, W, H, pyramid_gathers=1, **kw))
        assert ei.value.status == mrr.MRR_EINVAL
    fr = sg.gbuffer(0, W, H, 6, 2)
    ctx = mrr.mrr_create(make_cfg("ssao", 4, W, H, pyramid_gathers=1))
    dev = mrr.upload_frame(fr)
    b = mrr.mrr_batch_create()
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_render_batch(b, [ctx], [dev], [mrr.alloc_output(ctx, W, H)])
    assert ei.value.status == mrr.MRR_EUNSUPPORTED
    mrr.mrr_batch_destroy(b)
    mrr.mrr_destroy(ctx)


def test_ssao64_1080p_pyramid_full_size(mrr):
    """The 1920x1080 SSAO-64 workload with pyramid gathers in the launch configuration the
    benchmark times: the composite against the oracle over the whole frame, and level 0
    (which gathers at full resolution either way) equal to the default path's."""
    import torch
    wl = sg.WORKLOADS["ssao64_1080p"]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"])
    cfg = make_cfg("ssao", 4, W, H, samples=64, pyramid_gathers=1)
    ref = orc.render(fr, cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref["out"][..., 0]).max() <= TOL32
    mrr.mrr_destroy(ctx)
