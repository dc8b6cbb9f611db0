"""Mask tiles with no edge in their staged rows.  On the frame path such a tile writes its
constant levels directly (zeros at the blurred and disabled levels, ones and list entries at
the coarsest), instead of the general path's nesting, scans and per-texel tests.  Frames
with few objects (most tiles edge-free), every number of levels, and with level 1 disabled
(SSGI) must equal the staged calls bit for bit and the oracle within the bar (the all-sky
frame of the parity tests makes every tile edge-free)."""
import pytest

import scenegen as sg
from test_gpu_parity import check_frame, make_cfg

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


@pytest.mark.parametrize("effect,levels", [("ssao", 2), ("ssao", 3), ("ssao", 4), ("ssgi", 4), ("ssm", 4)])
def test_sparse_frames_match_staged_and_oracle(mrr, effect, levels):
    W, H = 520, 290  # ragged tiles at the right and bottom borders
    fr = sg.gbuffer(7, W, H, 3, 1, shadow_size=512 if effect == "ssm" else 0)
    check_frame(mrr, fr, make_cfg(effect, levels, W, H), "fp32", check_full=False)

