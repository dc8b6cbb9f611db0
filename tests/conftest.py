import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs the CUDA path")


def synthetic_frame(depth, normal, color=None, tan_half=None, near=0.1, far=50.0):
    """A Frame built from explicit planes, for closed-form pins."""
    import scenegen as sg
    depth = np.ascontiguousarray(depth, np.float32)
    H, W = depth.shape
    normal = np.ascontiguousarray(normal, np.float32)
    if color is None:
        color = np.zeros((H, W, 4), np.float32)
    cam = sg.camera(tan_half=sg.TAN_30 if tan_half is None else tan_half, near=near, far=far)
    return sg.Frame(W, H, depth, normal, np.ascontiguousarray(color, np.float32),
                    np.zeros((H, W), np.int32), cam)


def flat_normals(H, W, n=(0.0, 0.0, 1.0)):
    out = np.zeros((H, W, 4), np.float32)
    out[..., 0], out[..., 1], out[..., 2] = n
    return out
