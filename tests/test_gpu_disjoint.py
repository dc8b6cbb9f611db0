"""The disjoint-tile ablation (the decomposition without overlap that Sec. 3.1 rejects)
on the GPU against the oracle: stencils, blurred masks, labels and work lists bit-exact;
sub-images within the FP32 bar; the recomposition undefined (NaN) at exactly the oracle's
dead pixels and within the bar everywhere else; mrr_render equal to the staged calls."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from test_gpu_parity import TOL32, make_cfg, oracle_inputs, run_staged

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


@pytest.mark.parametrize("effect,W,H,levels", [("ssao", 203, 141, 4), ("ssao", 256, 256, 3), ("ssgi", 170, 100, 4),
                                               ("ssm", 196, 75, 4)])
def test_disjoint_tiles_match_the_oracle(mrr, effect, W, H, levels):
    import torch
    fr = sg.gbuffer(9, W, H, 20, 6, shadow_size=512 if effect == "ssm" else 0)
    cfg = make_cfg(effect, levels, W, H, disjoint=1)
    ref = orc.render(oracle_inputs(fr, "fp32"), cfg, "f32")
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    edges, lv, subs, out = run_staged(mrr, ctx, dev, W, H, levels)
    assert np.array_equal(edges.cpu().numpy(), ref["E"])
    for i in range(levels):
        assert np.array_equal(lv.stencil[i].cpu().numpy(), ref["S"][i]), i
        assert np.array_equal(lv.alpha[i].cpu().numpy().view(np.uint32), ref["a"][i].view(np.uint32)), i
        n = len(ref["lists"][i])
        assert lv.counts[i].item() == n
        assert np.array_equal(lv.worklist[i][:n].cpu().numpy().view(np.uint32), ref["lists"][i])
    assert np.array_equal(lv.label.cpu().numpy(), ref["label"])
    C = 3 if effect == "ssgi" else 1
    got = out.cpu().numpy()
    got = got if C == 1 else got[..., :3]
    exp = ref["out"][..., 0] if C == 1 else ref["out"]
    dead = np.isnan(exp)
    assert dead.any()                                    # the variant's dead pixels
    assert np.array_equal(np.isnan(got), dead)
    assert np.abs(got[~dead] - exp[~dead]).max() <= TOL32
    out2 = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out2)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), out2.cpu().numpy(), equal_nan=True)
    mrr.mrr_destroy(ctx)


def test_disjoint_tiles_are_single_frame_only(mrr):
    W, H = 64, 48
    cfg = make_cfg("ssao", 4, W, H, disjoint=1)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(sg.gbuffer(0, W, H, 4, 0))
    b = mrr.mrr_batch_create()
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_render_batch(b, [ctx], [dev], [mrr.alloc_output(ctx, W, H)])
    assert ei.value.status == mrr.MRR_EUNSUPPORTED
    mrr.mrr_batch_destroy(b)
    mrr.mrr_destroy(ctx)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_create(make_cfg("ssao", 4, W, H, disjoint=1, merge_mode=1))
