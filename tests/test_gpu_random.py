"""Seeded random configurations against the oracle: frame size, effect, number of levels
and which of them are enabled, blur variances, blend weights, edge thresholds, storage
precision and the optional stages (sub-image blur, step-wise or bilateral blending,
sample-count levels, pyramid gathers) drawn at random, each case checked stage by stage as the other parity tests do
(masks and lists bit-exact, sub-images and composite within the FP32 / FP16 bars,
mrr_render equal to the staged calls bit for bit)."""
import math

import numpy as np
import pytest

import scenegen as sg
from test_gpu_parity import check_frame, make_cfg
from test_gpu_samples import check_samples

pytestmark = pytest.mark.gpu

SIGMA2 = [0.3, 0.5, 0.924, 1.0, 1.848, 2.5, 3.696]   # blur radii ceil(3 sigma) from 2 to 6


@pytest.fixture(scope="module")
def mrr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


def draw(case):
    rng = np.random.default_rng(1000 + case)
    effect = ["ssao", "ssm", "ssgi"][case % 3]
    L = int(rng.integers(2, 5))
    W, H = int(rng.integers(1, 260)), int(rng.integers(1, 160))
    enabled = [1] * L
    for i in range(L - 1):
        if rng.random() < 0.25:
            enabled[i] = 0
    sigma2 = [float(rng.choice(SIGMA2)) for _ in range(L - 1)] + [0.0]
    weight = [float(rng.choice([0.5, 1.0, 4.0, 20.0, 100.0, 1000.0])) for _ in range(L - 1)] + [1.0]
    pad = 4 - L
    kw = dict(sigma2=sigma2 + [0.0] * pad, weight=weight + [0.0] * pad, enabled=enabled + [0] * pad,
              depth_rel=float(rng.uniform(0.02, 0.1)), normal_cos=float(rng.uniform(0.8, 0.97)))
    option = int(rng.integers(0, 4))            # 0 none, 1 blur, 2 step-wise or bilateral, 3 sample-count levels
    if option == 1 and any(enabled[1:L]):
        kw["blur"] = [0] + [int(enabled[i] and rng.random() < 0.7) for i in range(1, L)] + [0] * pad
    elif option == 2:
        kw["merge_mode"] = 1 if rng.random() < 0.5 else 2
    elif option == 3:
        kw["sample_levels"] = 1
    precision = "fp16" if rng.random() < 0.4 else "fp32"
    if effect != "ssm":
        kw["samples"] = int(rng.choice([8, 16, 24]))
    seed = int(rng.integers(0, 1 << 16))
    if effect == "ssao" and "sample_levels" not in kw and rng.random() < 0.5:
        kw["pyramid_gathers"] = 1
    return effect, L, W, H, precision, kw, seed


@pytest.mark.parametrize("case", range(24))
def test_random_configuration(mrr, case):
    effect, L, W, H, precision, kw, seed = draw(case)
    fr = sg.gbuffer(seed, W, H, 12, 4, shadow_size=256 if effect == "ssm" else 0)
    cfg = make_cfg(effect, L, W, H, precision, **kw)
    assert all(math.ceil(3 * math.sqrt(s)) <= 6 for s in cfg["sigma2"])
    if kw.get("sample_levels"):
        check_samples(mrr, fr, cfg, precision)
    else:
        check_frame(mrr, fr, cfg, precision, check_full=False)
