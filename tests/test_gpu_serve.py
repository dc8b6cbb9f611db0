"""Serving on the GPU: requests of mixed size and effect submitted together overlap on
the device (slots, batches) and every result equals the frame rendered alone."""
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


PREC = {"ssao": "fp32", "ssm": "fp32", "ssgi": "fp16"}


def _cfg(effect, W, H):
    kw = {}
    if effect == "ssm":
        kw.update(blocker_taps=sg.disk_taps(32, sg.BLOCKER_SEED), pcf_taps=sg.disk_taps(64, sg.PCF_SEED))
    else:
        n = 32
        kw.update(samples=n, kernel=sg.hemisphere_kernel(n), radius=0.5 if effect == "ssao" else 1.0)
    cfg = orc.default_config(effect, 4, **kw)
    cfg.update(precision=PREC[effect], max_width=W, max_height=H)
    return cfg


def test_mixed_requests_equal_frames_rendered_alone(mrr):
    import torch
    W, H = 480, 272
    cfgs = {e: _cfg(e, W, H) for e in ("ssao", "ssm", "ssgi")}
    srv = mrr.mrr_server_create(cfgs, slots=2)
    assert mrr.mrr_server_slots(srv) == 2
    jobs = [("ssao", 480, 272, 1), ("ssgi", 320, 180, 2), ("ssm", 400, 224, 3), ("ssao", 211, 97, 4),
            ("ssgi", 480, 272, 5), ("ssm", 480, 272, 6), ("ssao", 320, 180, 7), ("ssao", 480, 272, 1)]
    frames, outs, tickets = [], [], []
    for effect, w, h, seed in jobs:
        fr = sg.gbuffer(seed, w, h, 20, 6, shadow_size=512 if effect == "ssm" else 0)
        dev = mrr.upload_frame(fr, PREC[effect])
        ctx_like = mrr.Context(0, cfgs[effect])
        out = mrr.alloc_output(ctx_like, w, h)
        out.fill_(float("nan"))
        frames.append(dev)
        outs.append(out)
    torch.cuda.synchronize()
    for (effect, *_), dev, out in zip(jobs, frames, outs):
        tickets.append(mrr.mrr_submit(srv, effect, dev, out))
    for t in tickets:
        assert mrr.mrr_wait(srv, t, 30_000_000_000) == mrr.MRR_OK
    # alone, one context per effect, one frame at a time
    alone = {e: mrr.mrr_create(cfgs[e]) for e in cfgs}
    for (effect, w, h, _), dev, out in zip(jobs, frames, outs):
        ref = mrr.alloc_output(alone[effect], w, h)
        mrr.mrr_render(alone[effect], dev, ref)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), effect
    info = [mrr.mrr_request_info(srv, t) for t in tickets]
    assert all(i["device_ms"] > 0 for i in info)
    mrr.mrr_server_destroy(srv)
    for c in alone.values():
        mrr.mrr_destroy(c)


def test_graphs_are_reused_across_requests_with_fresh_buffers(mrr):
    """Waves of requests, every one with its own newly allocated inputs and output: the
    batches repeat topologies (the same contexts in the same order), so their graphs are
    updated in place rather than instantiated again, and every result still equals the
    frame rendered alone."""
    import torch
    W, H = 480, 272
    cfgs = {e: _cfg(e, W, H) for e in ("ssao", "ssgi")}
    srv = mrr.mrr_server_create(cfgs, slots=1, per_effect=2)
    alone = {e: mrr.mrr_create(cfgs[e]) for e in cfgs}
    sizes = [(480, 272), (320, 180), (400, 224), (211, 97)]
    for wave in range(4):
        jobs = [("ssao", *sizes[wave % 4]), ("ssao", *sizes[(wave + 1) % 4]), ("ssgi", *sizes[(wave + 2) % 4])]
        devs, outs = [], []
        for k, (effect, w, h) in enumerate(jobs):
            fr = sg.gbuffer(10 * wave + k, w, h, 20, 6)
            devs.append(mrr.upload_frame(fr, PREC[effect]))        # fresh device buffers
            o = mrr.alloc_output(mrr.Context(0, cfgs[effect]), w, h)
            o.fill_(float("nan"))
            outs.append(o)
        torch.cuda.synchronize()
        tickets = [mrr.mrr_submit(srv, e, d, o) for (e, _, _), d, o in zip(jobs, devs, outs)]
        for t in tickets:
            assert mrr.mrr_wait(srv, t, 30_000_000_000) == mrr.MRR_OK
        for (effect, w, h), d, o in zip(jobs, devs, outs):
            ref = mrr.alloc_output(alone[effect], w, h)
            mrr.mrr_render(alone[effect], d, ref)
            torch.cuda.synchronize()
            assert torch.equal(o, ref), (wave, effect)
    st = mrr.mrr_server_stats(srv)
    assert st["completed"] == 12
    assert st["graph_updates"] >= 1
    assert st["graph_instantiations"] + st["graph_updates"] == st["batches"]
    mrr.mrr_server_destroy(srv)
    for c in alone.values():
        mrr.mrr_destroy(c)
