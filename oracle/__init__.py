"""CPU oracle for the multi-resolution rendering method (arXiv 1906.04576).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product (the CUDA library
and its binding) never imports this package, and this package never imports the
product; both consume the seeded inputs made by ``scenegen``.

The arithmetic lives in ``oracle.cpp`` (plain C++, templated on float for the
parity oracle and on double for the FP64 reference).  This module only marshals
numpy arrays and composes the paper's three steps (Sec. 3): masks (Sec. 3.1),
sub-image rendering (Sec. 3.2 / 4.1) and blending (Sec. 4.2, Eq. (1)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

EFFECTS = {"ssao": 0, "ssm": 1, "ssgi": 2}

# Table 1 of the paper: (sigma_i^2, w_i) per sub-image i = 1..4 (full, 1/2, 1/4, 1/8).
# SSGI does not use the second sub-image ("--" in the table).
TABLE1 = {
    "ssao": [(0.924, 100.0), (1.848, 50.0), (3.696, 20.0), (0.0, 1.0)],
    "ssm": [(0.924, 1000.0), (1.848, 1000.0), (3.696, 1000.0), (0.0, 1.0)],
    "ssgi": [(0.924, 1000.0), None, (0.924, 100.0), (0.0, 1.0)],
}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so beside it (g++, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("effect", ctypes.c_int), ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("num_levels", ctypes.c_int),
        ("sigma2", ctypes.c_float * 4), ("weight", ctypes.c_float * 4), ("enabled", ctypes.c_int * 4),
        ("depth_rel", ctypes.c_float), ("normal_cos", ctypes.c_float), ("force_level0", ctypes.c_int),
        ("samples", ctypes.c_int), ("radius", ctypes.c_float), ("ao_bias", ctypes.c_float),
        ("gi_min_dist2", ctypes.c_float), ("kernel", ctypes.POINTER(ctypes.c_float)),
        ("blocker_samples", ctypes.c_int), ("pcf_samples", ctypes.c_int),
        ("blocker_taps", ctypes.POINTER(ctypes.c_float)), ("pcf_taps", ctypes.POINTER(ctypes.c_float)),
        ("light_size", ctypes.c_float), ("shadow_bias", ctypes.c_float), ("store_half", ctypes.c_int),
        ("cam", ctypes.c_float * 15), ("light", ctypes.c_float * 15), ("shadow_size", ctypes.c_int),
        ("blur", ctypes.c_int * 4), ("blur_depth_rel", ctypes.c_float), ("merge_mode", ctypes.c_int),
        ("sample_levels", ctypes.c_int), ("pyramid_gathers", ctypes.c_int), ("gather_level", ctypes.c_int),
        ("disjoint", ctypes.c_int),
    ]


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(Params)
        vp = ctypes.c_void_p
        ci = ctypes.c_int
        for suf in ("f32", "f64"):
            getattr(lib, f"orc_edges_{suf}").argtypes = [P, vp, vp, vp, vp]
            getattr(lib, f"orc_hard_shadow_{suf}").argtypes = [P, vp, vp, vp]
            getattr(lib, f"orc_masks_{suf}").argtypes = [P, vp, vp, vp, vp]
            getattr(lib, f"orc_shade_level_{suf}").argtypes = [P, vp, vp, vp, vp, ci, vp, ci, vp]
            getattr(lib, f"orc_shade_full_{suf}").argtypes = [P, vp, vp, vp, vp, vp]
            getattr(lib, f"orc_shade_pixel_{suf}").argtypes = [P, vp, vp, vp, vp, ci, ci, vp]
            getattr(lib, f"orc_view_pos_{suf}").argtypes = [P, ci, ci, ctypes.c_double, vp]
            getattr(lib, f"orc_make_basis_{suf}").argtypes = [vp, vp]
            getattr(lib, f"orc_merge_{suf}").argtypes = [P, vp, vp, vp, vp]
            getattr(lib, f"orc_blur_level_{suf}").argtypes = [P, vp, ci, vp, vp, vp]
            getattr(lib, f"orc_merge_stepwise_{suf}").argtypes = [P, vp, vp, vp, vp]
            getattr(lib, f"orc_merge_samples_{suf}").argtypes = [P, vp, vp, vp, vp]
            getattr(lib, f"orc_merge_disjoint_{suf}").argtypes = [P, vp, vp, vp]
            getattr(lib, f"orc_merge_bilateral_{suf}").argtypes = [P, vp, vp, vp, vp, vp]
            getattr(lib, f"orc_shade_blocks_{suf}").argtypes = [P, vp, vp, vp, vp, ci, vp, ci, vp]
        lib.orc_gauss_weights_f32.argtypes = [ctypes.c_double, vp]
        lib.orc_gauss_weights_f64.argtypes = [ctypes.c_double, vp]
        lib.orc_compact.argtypes = [ci, ci, vp, vp]
        lib.orc_compact.restype = ci
        lib.orc_round_to_half.argtypes = [ctypes.c_float]
        lib.orc_round_to_half.restype = ctypes.c_float
        lib.orc_level_dim.argtypes = [ci, ci]
        lib.orc_level_sample.argtypes = [ci, ci, ci]
        lib.orc_set_threads.argtypes = [ci]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    return _L().orc_num_threads()


def set_threads(n: int) -> None:
    _L().orc_set_threads(int(n))


def level_dim(n: int, level: int) -> int:
    return _L().orc_level_dim(n, level)


def level_sample(q: int, level: int, n: int) -> int:
    return _L().orc_level_sample(q, level, n)


def round_to_half(x: float) -> float:
    return _L().orc_round_to_half(float(x))


def gauss_weights(sigma2: float, dtype=np.float32) -> np.ndarray:
    g = np.zeros(64, dtype)
    fn = _L().orc_gauss_weights_f32 if dtype == np.float32 else _L().orc_gauss_weights_f64
    fn.restype = ctypes.c_int
    R = fn(float(sigma2), _ptr(g))
    return g[: 2 * R + 1].copy()


def default_config(effect: str, num_levels: int = 4, **kw) -> dict:
    """Paper parameters (Table 1, Sec. 4) plus our readings for what the paper leaves open."""
    rows = TABLE1[effect]
    if num_levels == 3:        # three levels: rows 1, 2 and the coarsest row
        rows = [rows[0], rows[1], rows[3]]
    sigma2, weight, enabled = [0.0] * 4, [0.0] * 4, [0] * 4
    for i, row in enumerate(rows[:num_levels]):
        if row is None:
            continue
        sigma2[i], weight[i] = row
        enabled[i] = 1
    cfg = dict(effect=effect, num_levels=num_levels, sigma2=sigma2, weight=weight, enabled=enabled,
               depth_rel=0.05, normal_cos=0.9, force_level0=0, samples=16, radius=0.5,
               ao_bias=0.0125, gi_min_dist2=0.01, kernel=None, blocker_samples=32, pcf_samples=64,
               blocker_taps=None, pcf_taps=None, light_size=0.5, shadow_bias=0.03, store_half=0,
               blur=[0, 0, 0, 0], blur_depth_rel=0.05, merge_mode=0, sample_levels=0, pyramid_gathers=0)
    cfg.update(kw)
    return cfg


class _Bound:
    """Params plus the numpy arrays its pointers refer to (kept alive together)."""

    def __init__(self, frame, cfg):
        p = Params()
        p.effect = EFFECTS[cfg["effect"]]
        p.width, p.height = frame.width, frame.height
        p.num_levels = cfg["num_levels"]
        for i in range(4):
            p.sigma2[i] = cfg["sigma2"][i]
            p.weight[i] = cfg["weight"][i]
            p.enabled[i] = int(cfg["enabled"][i])
        p.depth_rel, p.normal_cos = cfg["depth_rel"], cfg["normal_cos"]
        p.force_level0 = int(cfg.get("force_level0", 0))
        self.kernel = _f32(cfg.get("kernel"))
        self.btaps = _f32(cfg.get("blocker_taps"))
        self.ptaps = _f32(cfg.get("pcf_taps"))
        p.samples = cfg["samples"] if self.kernel is not None else 0
        p.radius, p.ao_bias, p.gi_min_dist2 = cfg["radius"], cfg["ao_bias"], cfg["gi_min_dist2"]
        p.kernel = ctypes.cast(_ptr(self.kernel), ctypes.POINTER(ctypes.c_float))
        p.blocker_samples = cfg["blocker_samples"] if self.btaps is not None else 0
        p.pcf_samples = cfg["pcf_samples"] if self.ptaps is not None else 0
        p.blocker_taps = ctypes.cast(_ptr(self.btaps), ctypes.POINTER(ctypes.c_float))
        p.pcf_taps = ctypes.cast(_ptr(self.ptaps), ctypes.POINTER(ctypes.c_float))
        p.light_size, p.shadow_bias = cfg["light_size"], cfg["shadow_bias"]
        p.store_half = int(cfg.get("store_half", 0))
        blur = cfg.get("blur", [0, 0, 0, 0])
        for i in range(4):
            p.blur[i] = int(blur[i])
        p.blur_depth_rel = cfg.get("blur_depth_rel", 0.05)
        p.merge_mode = int(cfg.get("merge_mode", 0))
        p.sample_levels = int(cfg.get("sample_levels", 0))
        p.pyramid_gathers = int(cfg.get("pyramid_gathers", 0))
        p.gather_level = 0
        p.disjoint = int(cfg.get("disjoint", 0))
        cam = frame.cam.as_array()
        for k in range(15):
            p.cam[k] = cam[k]
        if frame.light is not None:
            lc = frame.light.as_array()
            for k in range(15):
                p.light[k] = lc[k]
            p.shadow_size = frame.shadow_map.shape[0]
        self.p = p
        self.depth = _f32(frame.depth)
        self.normal = _f32(frame.normal)
        self.color = _f32(frame.color)
        self.smap = _f32(frame.shadow_map)

    @property
    def ref(self):
        return ctypes.byref(self.p)


def _suffix(precision):
    return {"f32": "f32", "f64": "f64"}[precision]


def _dtype(precision):
    return np.float32 if precision == "f32" else np.float64


def channels(cfg) -> int:
    return 3 if cfg["effect"] == "ssgi" else 1


def edges(frame, cfg, precision="f32") -> np.ndarray:
    b = _Bound(frame, cfg)
    E = np.zeros((frame.height, frame.width), np.uint8)
    getattr(_L(), f"orc_edges_{_suffix(precision)}")(b.ref, _ptr(b.depth), _ptr(b.normal), _ptr(b.smap), _ptr(E))
    return E


def hard_shadow(frame, cfg, precision="f32") -> np.ndarray:
    b = _Bound(frame, cfg)
    out = np.zeros((frame.height, frame.width), np.int32)
    getattr(_L(), f"orc_hard_shadow_{_suffix(precision)}")(b.ref, _ptr(b.depth), _ptr(b.smap), _ptr(out))
    return out


def _ptr_array(arrs):
    return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])


def masks(frame, cfg, E, precision="f32"):
    """Returns (a_i list, S_i list, label)."""
    b = _Bound(frame, cfg)
    L = cfg["num_levels"]
    dt = _dtype(precision)
    a = [np.zeros((level_dim(frame.height, i), level_dim(frame.width, i)), dt) for i in range(L)]
    S = [np.zeros((level_dim(frame.height, i), level_dim(frame.width, i)), np.uint8) for i in range(L)]
    label = np.zeros((frame.height, frame.width), np.uint8)
    E = np.ascontiguousarray(E, np.uint8)
    getattr(_L(), f"orc_masks_{_suffix(precision)}")(b.ref, _ptr(E), _ptr_array(a), _ptr_array(S), _ptr(label))
    return a, S, label


def compact(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, np.uint8)
    out = np.zeros(S.size, np.uint32)
    n = _L().orc_compact(S.shape[1], S.shape[0], _ptr(S), _ptr(out))
    return out[:n].copy()


def shade_level(frame, cfg, level, worklist, precision="f32"):
    b = _Bound(frame, cfg)
    dt = _dtype(precision)
    C = channels(cfg)
    Hi, Wi = level_dim(frame.height, level), level_dim(frame.width, level)
    c = np.full((Hi, Wi, C), np.nan, dt)
    wl = np.ascontiguousarray(worklist, np.uint32)
    getattr(_L(), f"orc_shade_level_{_suffix(precision)}")(
        b.ref, _ptr(b.depth), _ptr(b.normal), _ptr(b.color), _ptr(b.smap), level, _ptr(wl), len(wl), _ptr(c))
    return c


def shade_full(frame, cfg, precision="f32"):
    b = _Bound(frame, cfg)
    out = np.zeros((frame.height, frame.width, channels(cfg)), _dtype(precision))
    getattr(_L(), f"orc_shade_full_{_suffix(precision)}")(
        b.ref, _ptr(b.depth), _ptr(b.normal), _ptr(b.color), _ptr(b.smap), _ptr(out))
    return out


def shade_pixel(frame, cfg, x, y, precision="f64"):
    b = _Bound(frame, cfg)
    out = np.zeros(3, _dtype(precision))
    getattr(_L(), f"orc_shade_pixel_{_suffix(precision)}")(
        b.ref, _ptr(b.depth), _ptr(b.normal), _ptr(b.color), _ptr(b.smap), int(x), int(y), _ptr(out))
    return out[: channels(cfg)]


def view_pos(frame, cfg, x, y, d, precision="f64"):
    b = _Bound(frame, cfg)
    out = np.zeros(3, _dtype(precision))
    getattr(_L(), f"orc_view_pos_{_suffix(precision)}")(b.ref, int(x), int(y), float(d), _ptr(out))
    return out


def make_basis(n, precision="f64"):
    """The tangent frame the effects build around a unit normal n (Duff et al. 2017):
    rows t, b, n of a 3x3 array, in the oracle's precision."""
    nn = np.ascontiguousarray(n, np.float64).reshape(3)
    out = np.zeros(9, _dtype(precision))
    getattr(_L(), f"orc_make_basis_{_suffix(precision)}")(_ptr(nn), _ptr(out))
    return out.reshape(3, 3)


def level_config(cfg, level):
    """Sample-count levels (Sec. 6): level i keeps every 2^i-th entry of each sample table
    (entries 0, 2^i, 2 2^i, ...: ceil(n / 2^i) of n), so the thinned set spans the same
    range of sample lengths or disk radii as the full one."""
    out = dict(cfg)
    step = 1 << level
    if cfg.get("kernel") is not None:
        k = np.asarray(cfg["kernel"], np.float32).reshape(-1, 4)[::step]
        out.update(kernel=k, samples=len(k))
    for taps, count in (("blocker_taps", "blocker_samples"), ("pcf_taps", "pcf_samples")):
        if cfg.get(taps) is not None:
            t = np.asarray(cfg[taps], np.float32).reshape(-1, 2)[::step]
            out.update({taps: t, count: len(t)})
    return out


def shade_blocks(frame, cfg, level, worklist, precision="f32"):
    """Sample-count level `level`: every pixel of each listed texel's block at full
    resolution, with the level's thinned sample tables; [H][W][C], NaN elsewhere."""
    b = _Bound(frame, level_config(cfg, level))
    dt = _dtype(precision)
    c = np.full((frame.height, frame.width, channels(cfg)), np.nan, dt)
    wl = np.ascontiguousarray(worklist, np.uint32)
    getattr(_L(), f"orc_shade_blocks_{_suffix(precision)}")(
        b.ref, _ptr(b.depth), _ptr(b.normal), _ptr(b.color), _ptr(b.smap), level, _ptr(wl), len(wl), _ptr(c))
    return c


def merge(frame, cfg, a, S, c, precision="f32"):
    """Eq. (1): direct upsampling of every level (Sec. 4.2); with cfg["merge_mode"] = 1 the
    step-wise chain of Sec. 3.3, with 2 the direct upsampling with bilateral (depth-aware)
    taps; with cfg["sample_levels"] = 1 the full-resolution sub-images of sample-count
    levels (Sec. 6)."""
    b = _Bound(frame, cfg)
    dt = _dtype(precision)
    a = [np.ascontiguousarray(x, dt) for x in a]
    S = [np.ascontiguousarray(x, np.uint8) for x in S]
    c = [np.ascontiguousarray(x, dt) for x in c]
    out = np.zeros((frame.height, frame.width, channels(cfg)), dt)
    if cfg.get("disjoint", 0):
        getattr(_L(), f"orc_merge_disjoint_{_suffix(precision)}")(b.ref, _ptr_array(S), _ptr_array(c), _ptr(out))
        return out
    if cfg.get("merge_mode", 0) == 2 and not cfg.get("sample_levels", 0):
        getattr(_L(), f"orc_merge_bilateral_{_suffix(precision)}")(b.ref, _ptr(b.depth), _ptr_array(a),
                                                                   _ptr_array(S), _ptr_array(c), _ptr(out))
        return out
    if cfg.get("sample_levels", 0):
        fn = "orc_merge_samples"
    else:
        fn = "orc_merge_stepwise" if cfg.get("merge_mode", 0) == 1 else "orc_merge"
    getattr(_L(), f"{fn}_{_suffix(precision)}")(b.ref, _ptr_array(a), _ptr_array(S), _ptr_array(c), _ptr(out))
    return out


def blur_level(frame, cfg, level, S, c, precision="f32"):
    """Bilateral blur of sub-image `level` (Sec. 4.1) over its rendered texels S."""
    b = _Bound(frame, cfg)
    dt = _dtype(precision)
    S = np.ascontiguousarray(S, np.uint8)
    c = np.ascontiguousarray(c, dt)
    out = np.empty_like(c)
    getattr(_L(), f"orc_blur_level_{_suffix(precision)}")(b.ref, _ptr(b.depth), int(level), _ptr(S), _ptr(c),
                                                           _ptr(out))
    return out


def render(frame, cfg, precision="f32") -> dict:
    """The whole method (Sec. 3): edges -> masks -> work lists -> sub-images (blurred
    where cfg["blur"] asks, Sec. 4.1; full resolution with thinned samples above level 0
    when cfg["sample_levels"] is set, Sec. 6) -> Eq. (1)."""
    blur = cfg.get("blur", [0, 0, 0, 0])
    if cfg.get("sample_levels", 0) and (any(blur) or cfg.get("merge_mode", 0)):
        raise ValueError("sample-count levels take neither the sub-image blur nor step-wise blending")
    E = edges(frame, cfg, precision)
    a, S, label = masks(frame, cfg, E, precision)
    lists, c = [], []
    for i in range(cfg["num_levels"]):
        wl = compact(S[i])
        lists.append(wl)
        if cfg.get("sample_levels", 0) and i > 0:
            ci = shade_blocks(frame, cfg, i, wl, precision)
        else:
            ci = shade_level(frame, cfg, i, wl, precision)
        if blur[i]:
            ci = blur_level(frame, cfg, i, S[i], ci, precision)
        c.append(ci)
    out = merge(frame, cfg, a, S, c, precision)
    return dict(E=E, a=a, S=S, label=label, lists=lists, c=c, out=out)
