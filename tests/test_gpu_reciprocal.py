"""The effect kernels project sample points with their own reciprocal (the hardware
estimate refined by two Newton-Raphson steps, Markstein's form) instead of IEEE division.
The projections rely on it being the correctly rounded reciprocal wherever a sample depth
can lie, which this checks exhaustively: every float in [2^-64, 2^64) and its negative,
bit for bit against IEEE division."""
import pytest

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


def test_reciprocal_is_correctly_rounded_over_the_depth_range(mrr):
    lo, hi = 0x1F800000, 0x5F7FFFFF   # 2^-64 .. the largest float below 2^64
    assert mrr.mrr_check_reciprocal(lo, hi) == 0


def test_reciprocal_check_sees_a_range_edge(mrr):
    # subnormals are outside the claim: the hardware estimate flushes them, so the check
    # must report differences there (it is not vacuous)
    assert mrr.mrr_check_reciprocal(0x00200001, 0x00300000) > 0   # [2^-128, 2^-127.4]: finite reciprocals


def test_camera_outside_the_depth_range_is_rejected(mrr):
    import numpy as np
    import scenegen as sg
    import oracle as orc
    fr = sg.gbuffer(0, 16, 8, 1, 0)
    cfg = orc.default_config("ssao", 2, samples=4, kernel=sg.hemisphere_kernel(4), radius=0.5)
    cfg.update(precision="fp32", max_width=16, max_height=8)
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr)
    dev.cam = sg.camera(near=1e-30)
    out = mrr.alloc_output(ctx, 16, 8)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_render(ctx, dev, out)
    mrr.mrr_destroy(ctx)
