"""Seeded synthetic inputs for the multi-resolution rendering path.

This module makes INPUTS only: procedural scenes (ground plane y=0, axis-aligned
boxes, spheres), their G-buffers ray-cast in double precision and rounded once to
float, a light-space shadow map, and the seeded sample tables the lighting effects
draw (cosine-weighted hemisphere kernel, unit-disk taps).  It holds none of the
method's arithmetic; the CPU oracle and the CUDA path both consume what it returns.
The paper's test scenes (Sec. 5, "Office", "Hall", "Breakfast Room") are not
available; these seeded scenes stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.c")
_LIB = os.path.join(_HERE, "libscenegen.so")
_lib = None

# Camera of the synthetic scenes: eye (0,2,6) looking at the origin, vertical
# fov 60 deg (tan 30 deg = 1/sqrt(3)), near 0.1, far 50.
CAM_EYE = (0.0, 2.0, 6.0)
CAM_TARGET = (0.0, 0.0, 0.0)
TAN_30 = 1.0 / np.sqrt(3.0)
CAM_NEAR = 0.1
CAM_FAR = 50.0
# Light camera for soft shadow mapping: a square area light of side 0.5 centred at
# (4,8,4), looking at the origin; its shadow map uses a 60 deg square frustum.
LIGHT_EYE = (4.0, 8.0, 4.0)
LIGHT_NEAR = 4.0
LIGHT_FAR = 30.0
LIGHT_SIZE = 0.5

KERNEL_SEED = 0x5EED_A0
BLOCKER_SEED = 0x5EED_B1
PCF_SEED = 0x5EED_C2


def build(force: bool = False) -> str:
    """Compile scenegen.c into libscenegen.so beside it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d3 = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.POINTER(ctypes.c_int32)
        u64, ci, cd = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        lib.sg_gbuffer.argtypes = [u64, ci, ci, ci, ci, d3, d3, cd, cd, cd, fp, fp, fp, ip]
        lib.sg_gbuffer.restype = None
        lib.sg_pixel_world.argtypes = [u64, ci, ci, ci, ci, d3, d3, cd, cd, cd, ci, ci, d3]
        lib.sg_pixel_world.restype = ci
        lib.sg_shadow_map.argtypes = [u64, ci, ci, ci, d3, d3, cd, cd, cd, fp]
        lib.sg_shadow_map.restype = None
        lib.sg_camera.argtypes = [d3, d3, cd, cd, cd, fp]
        lib.sg_camera.restype = None
        lib.sg_hemisphere_kernel.argtypes = [u64, ci, fp]
        lib.sg_disk_taps.argtypes = [u64, ci, fp]
        lib.sg_poisson_stream.argtypes = [u64, ci, cd, ci, ctypes.POINTER(ctypes.c_double), ip]
        _lib = lib
    return _lib


def _d3(v):
    return (ctypes.c_double * 3)(*v)


def _fp(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


@dataclass
class Camera:
    """A pinhole camera as the floats handed to both consumers."""
    eye: np.ndarray
    right: np.ndarray
    up: np.ndarray
    forward: np.ndarray
    tan_half_fov: float
    near: float
    far: float

    def as_array(self) -> np.ndarray:
        return np.concatenate([self.eye, self.right, self.up, self.forward,
                               np.array([self.tan_half_fov, self.near, self.far], np.float32)]).astype(np.float32)


def camera(eye=CAM_EYE, target=CAM_TARGET, tan_half=TAN_30, near=CAM_NEAR, far=CAM_FAR) -> Camera:
    c = np.zeros(15, np.float32)
    _L().sg_camera(_d3(eye), _d3(target), float(tan_half), float(near), float(far), _fp(c))
    return Camera(c[0:3].copy(), c[3:6].copy(), c[6:9].copy(), c[9:12].copy(),
                  float(c[12]), float(c[13]), float(c[14]))


def light_camera() -> Camera:
    return camera(LIGHT_EYE, CAM_TARGET, TAN_30, LIGHT_NEAR, LIGHT_FAR)


@dataclass
class Frame:
    """One synthetic frame: G-buffer planes (row 0 = top) plus camera."""
    width: int
    height: int
    depth: np.ndarray    # float32 [H][W], linear view depth, sky = far
    normal: np.ndarray   # float32 [H][W][4], view-space unit normal, sky = 0
    color: np.ndarray    # float32 [H][W][4], direct light albedo*max(0,n.l)
    objid: np.ndarray    # int32 [H][W], -1 sky, 0 ground, 1.. objects
    cam: Camera
    seed: int = 0
    n_boxes: int = 0
    n_spheres: int = 0
    shadow_map: np.ndarray | None = None   # float32 [S][S] linear light depth
    light: Camera | None = None
    extra: dict = field(default_factory=dict)


def gbuffer(seed: int, width: int, height: int, n_boxes: int, n_spheres: int,
            eye=CAM_EYE, target=CAM_TARGET, tan_half=TAN_30, near=CAM_NEAR, far=CAM_FAR,
            shadow_size: int = 0) -> Frame:
    """Ray-cast the G-buffer of scene(seed); optionally the light's shadow map."""
    W, H = int(width), int(height)
    depth = np.empty((H, W), np.float32)
    normal = np.empty((H, W, 4), np.float32)
    color = np.empty((H, W, 4), np.float32)
    objid = np.empty((H, W), np.int32)
    _L().sg_gbuffer(seed, n_boxes, n_spheres, W, H, _d3(eye), _d3(target), float(tan_half),
                    float(near), float(far), _fp(depth), _fp(normal), _fp(color),
                    objid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    fr = Frame(W, H, depth, normal, color, objid, camera(eye, target, tan_half, near, far),
               seed, n_boxes, n_spheres)
    if shadow_size:
        fr.shadow_map = shadow_map(seed, n_boxes, n_spheres, shadow_size)
        fr.light = light_camera()
    return fr


def pixel_world(seed, width, height, n_boxes, n_spheres, x, y, eye=CAM_EYE, target=CAM_TARGET,
                tan_half=TAN_30, near=CAM_NEAR, far=CAM_FAR):
    """World-space hit point (double) of the ray through pixel (x,y), or None for sky."""
    out = (ctypes.c_double * 3)()
    ok = _L().sg_pixel_world(seed, n_boxes, n_spheres, width, height, _d3(eye), _d3(target),
                             float(tan_half), float(near), float(far), int(x), int(y), out)
    return np.array(list(out)) if ok else None


def shadow_map(seed: int, n_boxes: int, n_spheres: int, size: int,
               eye=LIGHT_EYE, target=CAM_TARGET, tan_half=TAN_30, near=LIGHT_NEAR,
               far=LIGHT_FAR) -> np.ndarray:
    sm = np.empty((size, size), np.float32)
    _L().sg_shadow_map(seed, n_boxes, n_spheres, size, _d3(eye), _d3(target), float(tan_half),
                       float(near), float(far), _fp(sm))
    return sm


def hemisphere_kernel(n: int, seed: int = KERNEL_SEED) -> np.ndarray:
    """Seeded cosine-weighted hemisphere samples (tangent frame), float32 [n][4]."""
    k = np.empty((n, 4), np.float32)
    _L().sg_hemisphere_kernel(seed, n, _fp(k))
    return k


def disk_taps(n: int, seed: int) -> np.ndarray:
    """Seeded uniform unit-disk points, float32 [n][2]."""
    t = np.empty((n, 2), np.float32)
    _L().sg_disk_taps(seed, n, _fp(t))
    return t


def poisson_stream(seed: int, n: int, rate: float, n_choices: int):
    """Exponential inter-arrival gaps (s) at `rate` per second and uniform picks."""
    gaps = np.empty(n, np.float64)
    pick = np.empty(n, np.int32)
    _L().sg_poisson_stream(seed, n, float(rate), n_choices,
                           gaps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           pick.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return gaps, pick


def to_half(a: np.ndarray) -> np.ndarray:
    """IEEE binary16 round-to-nearest-even of a float32 array (numpy's conversion)."""
    return a.astype(np.float16)


# Workloads of the paper's evaluation (Sec. 5), on synthetic scenes.
WORKLOADS = {
    # SSAO, 16 samples, radius 0.5, 3 levels, 256x256, 8 boxes
    "ssao16_256": dict(effect="ssao", width=256, height=256, n_boxes=8, n_spheres=0,
                       samples=16, radius=0.5, levels=3),
    # SSAO, 64 samples, radius 0.5, 4 levels, 1920x1080, 64 boxes + 16 spheres
    "ssao64_1080p": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                         samples=64, radius=0.5, levels=4),
    "ssao64_4k": dict(effect="ssao", width=3840, height=2160, n_boxes=64, n_spheres=16,
                      samples=64, radius=0.5, levels=4),
    # the same two with the bilateral blur of levels 1-3 (Sec. 4.1)
    "ssao64_1080p_blur": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                              samples=64, radius=0.5, levels=4, blur=(0, 1, 1, 1)),
    "ssao64_4k_blur": dict(effect="ssao", width=3840, height=2160, n_boxes=64, n_spheres=16,
                           samples=64, radius=0.5, levels=4, blur=(0, 1, 1, 1)),
    # the same two with the step-wise blending of Sec. 3.3
    "ssao64_1080p_step": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                              samples=64, radius=0.5, levels=4, merge_mode=1),
    "ssao64_4k_step": dict(effect="ssao", width=3840, height=2160, n_boxes=64, n_spheres=16,
                           samples=64, radius=0.5, levels=4, merge_mode=1),
    # with the direct merge's bilateral (depth-aware) taps (Sec. 3.3)
    "ssao64_1080p_bilateral": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                                   samples=64, radius=0.5, levels=4, merge_mode=2),
    "ssao64_4k_bilateral": dict(effect="ssao", width=3840, height=2160, n_boxes=64, n_spheres=16,
                                samples=64, radius=0.5, levels=4, merge_mode=2),
    # with pyramid gathers: levels above 0 gather depth from the level's point samples
    "ssao64_1080p_pyramid": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                                 samples=64, radius=0.5, levels=4, pyramid_gathers=1),
    "ssao64_4k_pyramid": dict(effect="ssao", width=3840, height=2160, n_boxes=64, n_spheres=16,
                              samples=64, radius=0.5, levels=4, pyramid_gathers=1),
    # and with sample-count levels (Sec. 6): levels above 0 at full resolution, fewer samples
    "ssao64_1080p_samples": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                                 samples=64, radius=0.5, levels=4, sample_levels=1),
    "ssao64_4k_samples": dict(effect="ssao", width=3840, height=2160, n_boxes=64, n_spheres=16,
                              samples=64, radius=0.5, levels=4, sample_levels=1),
    # the disjoint-tile ablation (complementary tiles without overlap, Sec. 3.1)
    "ssao64_1080p_disjoint": dict(effect="ssao", width=1920, height=1080, n_boxes=64, n_spheres=16,
                                  samples=64, radius=0.5, levels=4, disjoint=1),
    # soft shadows, 32 blocker + 64 PCF taps, 2048^2 shadow map, 4 levels, 2560x1440
    "ssm_1440p": dict(effect="ssm", width=2560, height=1440, n_boxes=64, n_spheres=16,
                      blocker_samples=32, pcf_samples=64, shadow_size=2048, levels=4),
    # SSGI, 32 samples, radius 1.0, levels 1, 1/4, 1/8 (the 1/2 level disabled), 3840x2160,
    # FP16 storage; batched with SSAO-64 on the same frame in one shading launch
    "ssgi32_4k": dict(effect="ssgi", width=3840, height=2160, n_boxes=64, n_spheres=16,
                      samples=32, radius=1.0, levels=4, precision="fp16",
                      batch_with=dict(effect="ssao", samples=64, radius=0.5, levels=4)),
    # serving mix: Poisson arrivals at 400/s, uniform over these resolutions x effects
    "serve_mix": dict(effect="mix", rate=400.0, requests=800,
                      resolutions=[(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)],
                      effects=[dict(effect="ssao", samples=64, radius=0.5, levels=4, precision="fp32"),
                               dict(effect="ssm", blocker_samples=32, pcf_samples=64, shadow_size=2048, levels=4,
                                    precision="fp32"),
                               dict(effect="ssgi", samples=32, radius=1.0, levels=4, precision="fp16")],
                      n_boxes=64, n_spheres=16, scenes_per_resolution=6, slots=4, per_effect=2),
}
