"""Batched rendering: several frames of different sizes, effects and storage
precisions in one pass with one persistent shading launch over a global queue; every
frame must equal the same frame rendered alone, bit for bit."""
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


def _cfg(effect, W, H, precision="fp32"):
    kw = {}
    if effect == "ssm":
        kw.update(blocker_taps=sg.disk_taps(32, sg.BLOCKER_SEED), pcf_taps=sg.disk_taps(64, sg.PCF_SEED))
    else:
        n = 64 if effect == "ssao" else 32
        kw.update(samples=n, kernel=sg.hemisphere_kernel(n), radius=0.5 if effect == "ssao" else 1.0)
    cfg = orc.default_config(effect, 4, store_half=int(precision == "fp16"), **kw)
    cfg.update(precision=precision, max_width=W, max_height=H)
    return cfg


JOBS = [("ssgi", 320, 180, "fp16", 1), ("ssao", 320, 180, "fp32", 1), ("ssao", 211, 97, "fp16", 2),
        ("ssm", 256, 144, "fp32", 3)]


def test_batch_equals_single_frames(mrr):
    import torch
    ctxs, frames, outs, refs = [], [], [], []
    for effect, W, H, prec, seed in JOBS:
        fr = sg.gbuffer(seed, W, H, 24, 6, shadow_size=512 if effect == "ssm" else 0)
        cfg = _cfg(effect, W, H, prec)
        ctx = mrr.mrr_create(cfg)
        dev = mrr.upload_frame(fr, prec)
        ref = mrr.alloc_output(ctx, W, H)
        mrr.mrr_render(ctx, dev, ref)
        ctxs.append(ctx)
        frames.append(dev)
        outs.append(mrr.alloc_output(ctx, W, H))
        refs.append(ref)
    b = mrr.mrr_batch_create()
    for rep in range(3):                 # capture, then graph replays
        for o in outs:
            o.fill_(float("nan"))
        mrr.mrr_render_batch(b, ctxs, frames, outs)
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
    t = mrr.mrr_batch_autotune(b, ctxs, frames)
    assert t["chunk"] in (256, 1024, 4096) and t["candidates"] == 6
    mrr.mrr_render_batch(b, ctxs, frames, outs)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    # a different subset and order re-captures
    mrr.mrr_render_batch(b, ctxs[::-1][:2], frames[::-1][:2], outs[::-1][:2])
    torch.cuda.synchronize()
    for o, r in zip(outs[::-1][:2], refs[::-1][:2]):
        assert torch.equal(o, r)
    mrr.mrr_batch_destroy(b)
    for c in ctxs:
        mrr.mrr_destroy(c)


def test_batch_frames_match_the_oracle(mrr):
    """Every frame of one batch (mixed sizes, effects and storage precisions, one
    persistent shading launch) against the oracle's composite on its own inputs (FP16
    storage: the oracle fed the same binary16 normals, shadow map and colour)."""
    import torch
    from test_gpu_parity import TOL16, TOL32, oracle_inputs
    ctxs, frames, outs, exps = [], [], [], []
    for effect, W, H, prec, seed in JOBS:
        fr = sg.gbuffer(seed, W, H, 24, 6, shadow_size=512 if effect == "ssm" else 0)
        cfg = _cfg(effect, W, H, prec)
        ref = orc.render(oracle_inputs(fr, prec), cfg, "f32")
        ctx = mrr.mrr_create(cfg)
        ctxs.append(ctx)
        frames.append(mrr.upload_frame(fr, prec))
        outs.append(mrr.alloc_output(ctx, W, H))
        exps.append((ref["out"], effect == "ssgi", TOL16 if prec == "fp16" else TOL32))
    b = mrr.mrr_batch_create()
    mrr.mrr_render_batch(b, ctxs, frames, outs)
    torch.cuda.synchronize()
    for o, (ro, gi, tol) in zip(outs, exps):
        got = o.cpu().numpy()
        got = got[..., :3] if gi else got
        exp = ro if gi else ro[..., 0]
        assert np.abs(got - exp).max() <= tol
    mrr.mrr_batch_destroy(b)
    for c in ctxs:
        mrr.mrr_destroy(c)


def test_batch_rejects_repeated_context(mrr):
    W, H = 64, 48
    fr = sg.gbuffer(0, W, H, 4, 0)
    cfg = _cfg("ssao", W, H)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    b = mrr.mrr_batch_create()
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_render_batch(b, [ctx, ctx], [dev, dev], [mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)])
    assert ei.value.status == mrr.MRR_EINVAL
    mrr.mrr_batch_destroy(b)
    mrr.mrr_destroy(ctx)
