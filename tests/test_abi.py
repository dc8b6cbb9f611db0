"""The C ABI library (libmrr.so) loads on a machine without a GPU and exports every
entry point include/mrr.h declares; argument validation answers before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mrr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mrr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(mrr_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_paper_stages():
    names = declared_functions()
    for n in ("mrr_create", "mrr_destroy", "mrr_edges", "mrr_masks", "mrr_shade_level", "mrr_upsample_merge",
              "mrr_render", "mrr_render_full", "mrr_level_dims", "mrr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(mrr):
    lib = mrr.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_level_dims_helper(mrr):
    assert mrr.mrr_level_dims(1920, 1080, 3) == (240, 135)
    assert mrr.mrr_level_dims(257, 129, 1) == (129, 65)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_level_dims(0, 10, 0)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_level_dims(10, 10, 4)


def test_invalid_arguments_are_rejected_before_any_launch(mrr):
    lib = mrr.lib()
    assert lib.mrr_create(None, None) == mrr.MRR_EINVAL
    h = ctypes.c_void_p()
    cfg = mrr.mrr_config()
    cfg.num_levels = 0
    assert lib.mrr_create(ctypes.byref(cfg), ctypes.byref(h)) == mrr.MRR_EINVAL and not h.value
    cfg.num_levels, cfg.enabled[0], cfg.max_width, cfg.max_height = 1, 1, 16, 16
    cfg.samples = 0          # SSAO needs a kernel
    assert lib.mrr_create(ctypes.byref(cfg), ctypes.byref(h)) == mrr.MRR_EINVAL
    cfg.samples, cfg.radius = 300, 0.5
    assert lib.mrr_create(ctypes.byref(cfg), ctypes.byref(h)) == mrr.MRR_EINVAL
    for fn, args in [("mrr_edges", (None, None, None, None)), ("mrr_masks", (None, None, None, None)),
                     ("mrr_render", (None, None, None, None)), ("mrr_render_full", (None, None, None, None)),
                     ("mrr_upsample_merge", (None, None, None, None, None)),
                     ("mrr_shade_level", (None, 0, None, None, None, None))]:
        assert getattr(lib, fn)(*args) == mrr.MRR_EINVAL, fn
