"""Parity at the sizes the benchmark workloads run, in the launch configuration they are
timed in (mrr_render's frame path), against the CPU oracle on the same seeded inputs:

* SSAO-64 at 3840x2160, FP32;
* soft shadows (32 blocker + 64 filter taps) at 2560x1440 with a 2048^2 shadow map, FP32;
* SSGI-32 at 3840x2160 with FP16 storage (the oracle fed the same binary16 inputs).

Each: the edge map, stencils and work lists of the staged path bit-exact over the whole
frame; the composite of the frame path against the oracle's whole-frame composite;
sampled full-resolution pixels of the plain kernel one by one; the RMSE gate of the
method against full-resolution shading.
"""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from test_gpu_parity import TOL16, TOL32, make_cfg, oracle_inputs, run_staged

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


def _check_workload(mrr, name, precision, cfg_kw, full_samples=300, rmse_gate=None):
    import torch
    wl = sg.WORKLOADS[name]
    W, H = wl["width"], wl["height"]
    fr = sg.gbuffer(0, W, H, wl["n_boxes"], wl["n_spheres"], shadow_size=wl.get("shadow_size", 0))
    cfg = make_cfg(wl["effect"], wl["levels"], W, H, precision, **cfg_kw)
    ofr = oracle_inputs(fr, precision)
    ref = orc.render(ofr, cfg, "f32")
    C = 3 if wl["effect"] == "ssgi" else 1
    tol = TOL16 if precision == "fp16" else TOL32
    ctx = mrr.mrr_create(cfg)
    dev = mrr.upload_frame(fr, precision)
    out = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    got = got if C == 1 else got[..., :3]
    exp = ref["out"][..., 0] if C == 1 else ref["out"]
    err = float(np.abs(got - exp).max())
    assert err <= tol, f"composite: {err}"
    L = wl["levels"]
    edges, levels, subs, _ = run_staged(mrr, ctx, dev, W, H, L)
    assert np.array_equal(edges.cpu().numpy(), ref["E"])
    for i in range(L):
        assert np.array_equal(levels.stencil[i].cpu().numpy(), ref["S"][i]), f"stencil {i}"
        assert np.array_equal(levels.alpha[i].cpu().numpy().view(np.uint32), ref["a"][i].view(np.uint32)), f"a {i}"
        n = len(ref["lists"][i])
        assert levels.counts[i].item() == n
        assert np.array_equal(levels.worklist[i][:n].cpu().numpy().view(np.uint32), ref["lists"][i])
    full = mrr.alloc_output(ctx, W, H)
    mrr.mrr_render_full(ctx, dev, full)
    torch.cuda.synchronize()
    g = full.cpu().numpy()
    g = g if C == 1 else g[..., :3]
    rng = np.random.default_rng(1)
    for _ in range(full_samples):
        x, y = int(rng.integers(W)), int(rng.integers(H))
        e = orc.shade_pixel(ofr, cfg, x, y, "f32")
        v = g[y, x] if C == 1 else g[y, x, :]
        assert np.abs(v - (e[0] if C == 1 else e)).max() <= TOL32, (x, y)
    if rmse_gate is not None:
        assert float(np.sqrt(np.mean((got - g) ** 2))) <= rmse_gate
    assert mrr.mrr_fault_flags(ctx) == 0
    mrr.mrr_destroy(ctx)


def test_ssao64_4k_full_size(mrr):
    _check_workload(mrr, "ssao64_4k", "fp32", dict(samples=64), rmse_gate=1e-2)


def test_ssm_1440p_full_size(mrr):
    _check_workload(mrr, "ssm_1440p", "fp32", dict())


def test_ssgi32_4k_fp16_full_size(mrr):
    _check_workload(mrr, "ssgi32_4k", "fp16", dict(samples=32, radius=1.0), full_samples=150)
