"""Level 0's alpha on the frame path.  There the list-aligned a_0 feeds only the level-0
blend's alpha = min(w_0 a_0, 1), and the mask kernel writes 1 instead of the exact a_0
for pixels within the Chebyshev radius r1 of an edge.  r1 is where one edge pixel already
makes fl(w_0 a_0) >= 1, and it depends on w_0.  With Table 1's level-0 variance (0.924,
radius 3) the weights 1, 10, 50, 1000 and 2e5 give r1 = none, 0, 1, 2 and 3.  Each frame
must equal the staged calls (which write the exact a_0 everywhere) bit for bit and the
oracle within the bar, and so must the same frames rendered as one batch."""
import numpy as np
import pytest

import scenegen as sg
from test_gpu_parity import check_frame, make_cfg

pytestmark = pytest.mark.gpu

WEIGHTS = [1.0, 10.0, 50.0, 1000.0, 2.0e5]


@pytest.fixture(scope="module")
def mrr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


def _cfg(effect, w0, W, H, precision="fp32"):
    kw = dict(weight=[w0, 1000.0, 100.0, 1.0]) if effect == "ssao" else dict(weight=[w0, 0.0, 100.0, 1.0])
    return make_cfg(effect, 4, W, H, precision, **kw)


@pytest.mark.parametrize("w0", WEIGHTS)
@pytest.mark.parametrize("effect", ["ssao", "ssgi"])
def test_level0_alpha_shortcut_matches_staged_and_oracle(mrr, effect, w0):
    W, H = 203, 141
    fr = sg.gbuffer(4, W, H, 20, 6)
    check_frame(mrr, fr, _cfg(effect, w0, W, H), "fp32", check_full=False)


def test_level0_alpha_shortcut_in_a_batch(mrr):
    import torch
    W, H = 160, 96
    ctxs, frames, refs, outs = [], [], [], []
    for k, w0 in enumerate(WEIGHTS):
        fr = sg.gbuffer(10 + k, W, H, 16, 4)
        ctx = mrr.mrr_create(_cfg("ssao", w0, W, H))
        dev = mrr.upload_frame(fr)
        ref = mrr.alloc_output(ctx, W, H)
        mrr.mrr_render(ctx, dev, ref)
        ctxs.append(ctx)
        frames.append(dev)
        refs.append(ref)
        outs.append(mrr.alloc_output(ctx, W, H))
    b = mrr.mrr_batch_create()
    mrr.mrr_render_batch(b, ctxs, frames, outs)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    mrr.mrr_batch_destroy(b)
    for c in ctxs:
        mrr.mrr_destroy(c)
