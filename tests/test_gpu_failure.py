"""Failure detection on the GPU without a GPU fault: the bounded wait the TMA edge kernel
uses on its tile loads is made to run out (an mbarrier phase that expects bytes no copy
will bring), records its bit in the context's fault word after about a second, and
returns; the context then renders exactly as before."""
import time

import numpy as np
import pytest

import scenegen as sg
from test_gpu_parity import make_cfg

pytestmark = pytest.mark.gpu

FAULT_EDGES_WAIT, FAULT_CHECK_WAIT = 1 << 0, 1 << 30


@pytest.fixture(scope="module")
def mrr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


def test_unanswered_wait_times_out_and_context_stays_usable(mrr):
    import torch
    W, H = 256, 144
    fr = sg.gbuffer(3, W, H, 16, 4)
    ctx = mrr.mrr_create(make_cfg("ssao", 4, W, H, samples=16))
    dev = mrr.upload_frame(fr)
    before, after = mrr.alloc_output(ctx, W, H), mrr.alloc_output(ctx, W, H)
    mrr.mrr_render(ctx, dev, before)
    assert mrr.mrr_fault_flags(ctx) == 0
    t0 = time.perf_counter()
    flags = mrr.mrr_check_wait_timeout(ctx)
    dt = time.perf_counter() - t0
    assert flags == FAULT_CHECK_WAIT                  # the wait gave up and said so
    assert 0.2 < dt < 30.0                            # bounded: about a second of SM clocks
    assert mrr.mrr_fault_flags(ctx, clear=True) == FAULT_CHECK_WAIT
    assert mrr.mrr_fault_flags(ctx) == 0
    mrr.mrr_render(ctx, dev, after)                   # the context still works, bit for bit
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    assert mrr.mrr_fault_flags(ctx) & FAULT_EDGES_WAIT == 0
    mrr.mrr_destroy(ctx)
