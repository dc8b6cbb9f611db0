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
