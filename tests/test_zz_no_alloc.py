"""mrr_masks_static: the mask stage for callers that cannot allocate device memory.

Such callers (code inside an engine that owns every device allocation, or one that
runs within a fixed memory budget) cannot create a context, because mrr_create
allocates pools.  mrr_masks_static needs no context and keeps its compaction scratch
in a fixed array inside the library.  This file is collected last so that a failure
here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg

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


def _levels_equal(a, b, L):
    for i in range(L):
        assert np.array_equal(a.alpha[i].cpu().numpy().view(np.uint32), b.alpha[i].cpu().numpy().view(np.uint32))
        assert np.array_equal(a.stencil[i].cpu().numpy(), b.stencil[i].cpu().numpy())
        n = int(a.counts[i].item())
        assert n == int(b.counts[i].item())
        assert np.array_equal(a.worklist[i][:n].cpu().numpy(), b.worklist[i][:n].cpu().numpy())
    assert np.array_equal(a.label.cpu().numpy(), b.label.cpu().numpy())


@pytest.mark.parametrize("effect,W,H", [("ssao", 1920, 1080), ("ssgi", 203, 141)])
def test_static_masks_match_mrr_masks_twice(mrr, effect, W, H):
    import torch
    kernel = sg.hemisphere_kernel(16)
    cfg = orc.default_config(effect, 4, samples=16, kernel=kernel)
    cfg.update(max_width=W, max_height=H)
    ctx = mrr.mrr_create(cfg)
    for seed in (3, 4):                       # two calls in a row, different frames
        fr = sg.gbuffer(seed, W, H, 32, 8)
        dev = mrr.upload_frame(fr)
        edges = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        mrr.mrr_edges(ctx, dev, edges)
        ref = mrr.alloc_levels(W, H, 4)
        mrr.mrr_masks(ctx, edges, ref)
        got = mrr.alloc_levels(W, H, 4)
        for lv in (got,):                     # poison the outputs first
            for t in lv.alpha + lv.stencil + lv.worklist:
                t.fill_(0x7F if t.dtype != torch.float32 else float("nan"))
        mrr.mrr_masks_static(cfg, edges, got)
        torch.cuda.synchronize()
        _levels_equal(got, ref, 4)
    mrr.mrr_destroy(ctx)


@pytest.mark.parametrize("case", ["sigma2_r4", "sigma2_r6", "three_levels", "force_level0"])
def test_static_masks_match_mrr_masks_other_patterns(mrr, case):
    """Patterns outside Table 1's: the generic mask kernel (level-0 radius 4, where the
    context uses its table of window sums and this call sums the taps, and radius 6),
    three levels, and every pixel forced to level 0."""
    import torch
    W, H = 257, 129
    kernel = sg.hemisphere_kernel(16)
    if case == "three_levels":
        cfg = orc.default_config("ssao", 3, samples=16, kernel=kernel)
    else:
        cfg = orc.default_config("ssao", 4, samples=16, kernel=kernel)
    if case == "sigma2_r4":
        cfg["sigma2"] = [1.5, 1.848, 3.696, 0.0]     # R_0 = ceil(3 sqrt(1.5)) = 4
    elif case == "sigma2_r6":
        cfg["sigma2"] = [3.5, 1.2, 2.0, 0.0]         # R = 6, 4, 5
    elif case == "force_level0":
        cfg["force_level0"] = 1
    L = cfg["num_levels"]
    cfg.update(max_width=W, max_height=H)
    ctx = mrr.mrr_create(cfg)
    for seed in (5, 6):
        fr = sg.gbuffer(seed, W, H, 12, 4)
        dev = mrr.upload_frame(fr)
        edges = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        mrr.mrr_edges(ctx, dev, edges)
        ref = mrr.alloc_levels(W, H, L)
        mrr.mrr_masks(ctx, edges, ref)
        got = mrr.alloc_levels(W, H, L)
        for t in got.alpha + got.stencil + got.worklist:
            t.fill_(0x7F if t.dtype != torch.float32 else float("nan"))
        mrr.mrr_masks_static(cfg, edges, got)
        torch.cuda.synchronize()
        _levels_equal(got, ref, L)
    mrr.mrr_destroy(ctx)


def test_static_masks_reject_non_positive_variance(mrr):
    import torch
    cfg = orc.default_config("ssao", 4, samples=16, kernel=sg.hemisphere_kernel(16))
    cfg["sigma2"] = [0.924, 0.0, 3.696, 0.0]        # a blurred level with sigma^2 = 0
    W, H = 64, 48
    cfg.update(max_width=W, max_height=H)
    edges = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    lv = mrr.alloc_levels(W, H, 4)
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_masks_static(cfg, edges, lv)
    assert ei.value.status == mrr.MRR_EINVAL


def test_static_masks_check_the_edge_tensor(mrr):
    import torch
    cfg = orc.default_config("ssao", 4, samples=16, kernel=sg.hemisphere_kernel(16))
    W, H = 64, 48
    lv = mrr.alloc_levels(W, H, 4)
    for bad in (torch.zeros((W, H), dtype=torch.uint8, device="cuda"),       # transposed
                torch.zeros((H, W), dtype=torch.float32, device="cuda"),     # wrong type
                torch.zeros((H, W), dtype=torch.uint8)):                     # host memory
        with pytest.raises(ValueError):
            mrr.mrr_masks_static(cfg, bad, lv)


def test_static_masks_reject_frames_beyond_the_scratch(mrr):
    import torch
    cfg = orc.default_config("ssao", 4, samples=16, kernel=sg.hemisphere_kernel(16))
    W, H = 4097, 8
    cfg.update(max_width=W, max_height=H)
    edges = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    lv = mrr.alloc_levels(W, H, 4)
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_masks_static(cfg, edges, lv)
    assert ei.value.status == mrr.MRR_EINVAL
