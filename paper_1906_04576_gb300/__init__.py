"""Python binding of libmrr, the CUDA (sm_103a) multi-resolution rendering library.

Argument marshalling only: every stage runs in libmrr's kernels.  PyTorch supplies
device memory and streams.  The functions carry the C names of include/mrr.h:

    mrr_create(cfg) -> Context          mrr_destroy(ctx)
    mrr_edges(ctx, frame, edges)        mrr_masks(ctx, edges, levels)
    mrr_shade_level(ctx, level, frame, levels, c)
    mrr_shade_levels(ctx, frame, levels, c_list)
    mrr_upsample_merge(ctx, levels, c_list, out)
    mrr_render(ctx, frame, out)         mrr_render_full(ctx, frame, out)
    mrr_render_host(ctx, host_frame, out_host)
    mrr_level_dims(W, H, level)         mrr_last_error(ctx)
    mrr_autotune(ctx, frame)            mrr_kernel_launches()
    mrr_batch_create() -> Batch         mrr_batch_destroy(b)
    mrr_render_batch(b, ctxs, frames, outs)   mrr_batch_autotune(b, ctxs, frames)
    mrr_masks_static(cfg, edges, levels)
    mrr_server_create(cfgs) -> Server   mrr_submit / mrr_poll / mrr_wait / mrr_request_info / mrr_release
    mrr_server_stats(s)

Importing raises if libmrr.so has not been built (``__graft_entry__.build()`` or
``python paper_1906_04576_gb300/_build.py``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmrr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmrr.so not built at {LIB_PATH}; run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

MRR_OK, MRR_EINVAL, MRR_ENOMEM, MRR_ECUDA, MRR_EBUSY, MRR_ETIMEDOUT, MRR_EUNSUPPORTED = range(7)
STATUS_NAMES = ["MRR_OK", "MRR_EINVAL", "MRR_ENOMEM", "MRR_ECUDA", "MRR_EBUSY", "MRR_ETIMEDOUT",
                "MRR_EUNSUPPORTED"]
MRR_SSAO, MRR_SSM, MRR_SSGI = 0, 1, 2
MRR_FP32, MRR_FP16 = 0, 1
MAX_LEVELS, MAX_SAMPLES, MAX_TAPS = 4, 256, 128
EFFECTS = {"ssao": MRR_SSAO, "ssm": MRR_SSM, "ssgi": MRR_SSGI}

F4 = ctypes.c_float * 4
I4 = ctypes.c_int * 4


class mrr_config(ctypes.Structure):
    _fields_ = [
        ("effect", ctypes.c_int), ("precision", ctypes.c_int), ("num_levels", ctypes.c_int),
        ("sigma2", F4), ("weight", F4), ("enabled", I4),
        ("depth_rel", ctypes.c_float), ("normal_cos", ctypes.c_float), ("force_level0", ctypes.c_int),
        ("samples", ctypes.c_int), ("radius", ctypes.c_float), ("ao_bias", ctypes.c_float),
        ("gi_min_dist2", ctypes.c_float), ("kernel", ctypes.POINTER(ctypes.c_float)),
        ("blocker_samples", ctypes.c_int), ("pcf_samples", ctypes.c_int),
        ("blocker_taps", ctypes.POINTER(ctypes.c_float)), ("pcf_taps", ctypes.POINTER(ctypes.c_float)),
        ("light_size", ctypes.c_float), ("shadow_bias", ctypes.c_float),
        ("max_width", ctypes.c_int), ("max_height", ctypes.c_int),
        ("lanes_per_texel", ctypes.c_int), ("lanes_per_pixel", ctypes.c_int), ("no_graph", ctypes.c_int),
        ("blur", I4), ("blur_depth_rel", ctypes.c_float), ("merge_mode", ctypes.c_int),
        ("sample_levels", ctypes.c_int), ("pyramid_gathers", ctypes.c_int), ("disjoint", ctypes.c_int),
    ]


class mrr_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("forward", ctypes.c_float * 3), ("tan_half_fov", ctypes.c_float),
                ("near_plane", ctypes.c_float), ("far_plane", ctypes.c_float)]


class mrr_gbuffer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("depth", ctypes.c_void_p),
                ("normal", ctypes.c_void_p), ("color", ctypes.c_void_p), ("shadow_map", ctypes.c_void_p),
                ("shadow_size", ctypes.c_int), ("cam", mrr_camera), ("light", mrr_camera)]


class mrr_levels(ctypes.Structure):
    _fields_ = [("num_levels", ctypes.c_int), ("width", I4), ("height", I4),
                ("alpha", ctypes.c_void_p * 4), ("stencil", ctypes.c_void_p * 4),
                ("worklist", ctypes.c_void_p * 4), ("counts", ctypes.c_void_p), ("label", ctypes.c_void_p)]


class mrr_tuning(ctypes.Structure):
    _fields_ = [("lanes_per_texel", ctypes.c_int), ("grid_multiplier", ctypes.c_int),
                ("lanes_per_pixel", ctypes.c_int), ("shade_levels_ms", ctypes.c_float),
                ("shade_full_ms", ctypes.c_float), ("candidates", ctypes.c_int)]


class mrr_server_config(ctypes.Structure):
    _fields_ = [("effect_cfg", mrr_config * 3), ("effect_enabled", ctypes.c_int * 3), ("slots", ctypes.c_int),
                ("hbm_reserve", ctypes.c_size_t), ("max_queue", ctypes.c_int), ("mock_device_us", ctypes.c_int),
                ("per_effect", ctypes.c_int), ("direct_launches", ctypes.c_int)]


class mrr_server_stats_t(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("graph_instantiations", ctypes.c_uint64), ("graph_updates", ctypes.c_uint64)]


class mrr_request(ctypes.Structure):
    _fields_ = [("effect", ctypes.c_int), ("frame", mrr_gbuffer), ("out_dev", ctypes.c_void_p)]


class mrr_request_info_t(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("result", ctypes.c_int), ("submit_ns", ctypes.c_int64),
                ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64), ("device_ms", ctypes.c_float)]


class mrr_batch_tuning(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int), ("grid_multiplier", ctypes.c_int), ("shade_ms", ctypes.c_float),
                ("candidates", ctypes.c_int)]


_vp = ctypes.c_void_p
_lib.mrr_batch_create.argtypes = [ctypes.POINTER(_vp)]
_lib.mrr_batch_create.restype = ctypes.c_int
_lib.mrr_batch_destroy.argtypes = [_vp]
_lib.mrr_batch_destroy.restype = None
_lib.mrr_render_batch.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(mrr_gbuffer), ctypes.POINTER(_vp),
                                  ctypes.c_int, _vp]
_lib.mrr_render_batch.restype = ctypes.c_int
_lib.mrr_batch_autotune.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(mrr_gbuffer), ctypes.c_int, _vp,
                                    ctypes.POINTER(mrr_batch_tuning)]
_lib.mrr_batch_autotune.restype = ctypes.c_int
_lib.mrr_batch_last_error.argtypes = [_vp]
_lib.mrr_batch_last_error.restype = ctypes.c_char_p
_lib.mrr_server_create.argtypes = [ctypes.POINTER(mrr_server_config), ctypes.POINTER(_vp)]
_lib.mrr_server_create.restype = ctypes.c_int
_lib.mrr_server_destroy.argtypes = [_vp]
_lib.mrr_server_destroy.restype = None
_lib.mrr_server_slots.argtypes = [_vp]
_lib.mrr_server_slots.restype = ctypes.c_int
_lib.mrr_submit.argtypes = [_vp, ctypes.POINTER(mrr_request), ctypes.POINTER(ctypes.c_uint64)]
_lib.mrr_submit.restype = ctypes.c_int
_lib.mrr_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
_lib.mrr_poll.restype = ctypes.c_int
_lib.mrr_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int64]
_lib.mrr_wait.restype = ctypes.c_int
_lib.mrr_request_info.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(mrr_request_info_t)]
_lib.mrr_server_stats.argtypes = [_vp, ctypes.POINTER(mrr_server_stats_t)]
_lib.mrr_server_stats.restype = ctypes.c_int
_lib.mrr_request_info.restype = ctypes.c_int
_lib.mrr_release.argtypes = [_vp, ctypes.c_uint64]
_lib.mrr_release.restype = ctypes.c_int
_lib.mrr_autotune.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), _vp, ctypes.POINTER(mrr_tuning)]
_lib.mrr_autotune.restype = ctypes.c_int
_lib.mrr_level_dims.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]
_lib.mrr_create.argtypes = [ctypes.POINTER(mrr_config), ctypes.POINTER(_vp)]
_lib.mrr_destroy.argtypes = [_vp]
_lib.mrr_destroy.restype = None
_lib.mrr_last_error.argtypes = [_vp]
_lib.mrr_last_error.restype = ctypes.c_char_p
_lib.mrr_edges.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), _vp, _vp]
_lib.mrr_masks.argtypes = [_vp, _vp, ctypes.POINTER(mrr_levels), _vp]
_lib.mrr_shade_level.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(mrr_gbuffer), ctypes.POINTER(mrr_levels), _vp, _vp]
_lib.mrr_upsample_merge.argtypes = [_vp, ctypes.POINTER(mrr_levels), ctypes.POINTER(_vp), _vp, _vp]
_lib.mrr_upsample_merge_bilateral.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), ctypes.POINTER(mrr_levels),
                                              ctypes.POINTER(_vp), _vp, _vp]
_lib.mrr_blur_level.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(mrr_gbuffer), ctypes.POINTER(mrr_levels), _vp, _vp,
                                _vp]
_lib.mrr_shade_levels.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), ctypes.POINTER(mrr_levels), ctypes.POINTER(_vp), _vp]
_lib.mrr_masks_static.argtypes = [ctypes.POINTER(mrr_config), _vp, ctypes.POINTER(mrr_levels), _vp]
_lib.mrr_masks_static.restype = ctypes.c_int
_lib.mrr_kernel_launches.argtypes = []
_lib.mrr_kernel_launches.restype = ctypes.c_uint64
_lib.mrr_fault_flags.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
_lib.mrr_check_wait_timeout.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint32)]
_lib.mrr_check_reciprocal.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]
_lib.mrr_render.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), _vp, _vp]
_lib.mrr_render_full.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), _vp, _vp]
_lib.mrr_trace_shading.argtypes = [_vp, _vp, _vp]
_lib.mrr_trace_shading.restype = ctypes.c_int
_lib.mrr_render_host.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), _vp, _vp]
_lib.mrr_render_host_async.argtypes = [_vp, ctypes.POINTER(mrr_gbuffer), _vp]
_lib.mrr_render_host_async.restype = ctypes.c_int
_lib.mrr_render_host_wait.argtypes = [_vp]
_lib.mrr_render_host_wait.restype = ctypes.c_int
for _fn in ("mrr_level_dims", "mrr_create", "mrr_edges", "mrr_masks", "mrr_shade_level", "mrr_shade_levels",
            "mrr_upsample_merge", "mrr_upsample_merge_bilateral", "mrr_blur_level",
            "mrr_render", "mrr_render_full", "mrr_render_host"):
    getattr(_lib, _fn).restype = ctypes.c_int


class MrrError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")


def lib() -> ctypes.CDLL:
    return _lib


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


@dataclass
class Context:
    handle: int
    config: dict
    _keep: list = field(default_factory=list)

    @property
    def channels(self) -> int:
        return 4 if self.config["effect"] == "ssgi" else 1

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _lib.mrr_destroy(h)
            except Exception:
                pass
            self.handle = 0


def _check(ctx, st):
    if st != MRR_OK:
        msg = _lib.mrr_last_error(ctx.handle if ctx is not None else None)
        raise MrrError(st, msg.decode() if msg else "")


def mrr_level_dims(width: int, height: int, level: int):
    wi, hi = ctypes.c_int(), ctypes.c_int()
    st = _lib.mrr_level_dims(width, height, level, ctypes.byref(wi), ctypes.byref(hi))
    if st != MRR_OK:
        raise MrrError(st, "mrr_level_dims")
    return wi.value, hi.value


def make_config(cfg: dict) -> tuple[mrr_config, list]:
    """mrr_config from a dict (keys as in the C struct; effect as 'ssao'/'ssm'/'ssgi')."""
    import numpy as np
    c = mrr_config()
    keep = []
    c.effect = EFFECTS[cfg["effect"]]
    c.precision = MRR_FP16 if cfg.get("precision", "fp32") == "fp16" else MRR_FP32
    c.num_levels = cfg["num_levels"]
    for i in range(4):
        c.sigma2[i] = cfg["sigma2"][i]
        c.weight[i] = cfg["weight"][i]
        c.enabled[i] = int(cfg["enabled"][i])
    c.depth_rel = cfg.get("depth_rel", 0.05)
    c.normal_cos = cfg.get("normal_cos", 0.9)
    c.force_level0 = int(cfg.get("force_level0", 0))

    def table(name, n_key, cols):
        arr = cfg.get(name)
        if arr is None:
            return None, 0
        a = np.ascontiguousarray(arr, dtype=np.float32).reshape(-1, cols)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.shape[0]

    c.kernel, n = table("kernel", "samples", 4)
    c.samples = n
    c.radius = cfg.get("radius", 0.5)
    c.ao_bias = cfg.get("ao_bias", 0.0125)
    c.gi_min_dist2 = cfg.get("gi_min_dist2", 0.01)
    c.blocker_taps, c.blocker_samples = table("blocker_taps", "blocker_samples", 2)
    c.pcf_taps, c.pcf_samples = table("pcf_taps", "pcf_samples", 2)
    c.light_size = cfg.get("light_size", 0.5)
    c.shadow_bias = cfg.get("shadow_bias", 0.03)
    c.max_width = cfg["max_width"]
    c.max_height = cfg["max_height"]
    c.lanes_per_texel = int(cfg.get("lanes_per_texel", 0))
    c.lanes_per_pixel = int(cfg.get("lanes_per_pixel", 0))
    c.no_graph = int(cfg.get("no_graph", 0))
    blur = cfg.get("blur", [0, 0, 0, 0])
    for i in range(4):
        c.blur[i] = int(blur[i])
    c.blur_depth_rel = cfg.get("blur_depth_rel", 0.05)
    c.merge_mode = int(cfg.get("merge_mode", 0))
    c.sample_levels = int(cfg.get("sample_levels", 0))
    c.pyramid_gathers = int(cfg.get("pyramid_gathers", 0))
    c.disjoint = int(cfg.get("disjoint", 0))
    return c, keep


def mrr_create(cfg: dict) -> Context:
    c, keep = make_config(cfg)
    h = _vp()
    st = _lib.mrr_create(ctypes.byref(c), ctypes.byref(h))
    if st != MRR_OK:
        raise MrrError(st, "mrr_create")
    return Context(h.value, dict(cfg))


def mrr_destroy(ctx: Context) -> None:
    if ctx.handle:
        _lib.mrr_destroy(ctx.handle)
        ctx.handle = 0


def mrr_last_error(ctx: Context) -> str:
    return _lib.mrr_last_error(ctx.handle).decode()


def _camera(cam) -> mrr_camera:
    m = mrr_camera()
    for k in range(3):
        m.eye[k], m.right[k], m.up[k], m.forward[k] = cam.eye[k], cam.right[k], cam.up[k], cam.forward[k]
    m.tan_half_fov, m.near_plane, m.far_plane = cam.tan_half_fov, cam.near, cam.far
    return m


@dataclass
class DeviceFrame:
    """A G-buffer resident on the device (torch tensors) plus its cameras."""
    width: int
    height: int
    depth: torch.Tensor                   # float32 [H][W]
    normal: torch.Tensor                  # float32 [H][W][4] or float16 [H][W][4]
    cam: object
    color: torch.Tensor | None = None     # float16 [H][W][4]
    shadow_map: torch.Tensor | None = None  # float32 [S][S] (light depth stays FP32 in both precisions)
    light: object = None

    def struct(self) -> mrr_gbuffer:
        g = mrr_gbuffer()
        g.width, g.height = self.width, self.height
        g.depth = _ptr(self.depth)
        g.normal = _ptr(self.normal)
        g.color = _ptr(self.color)
        g.shadow_map = _ptr(self.shadow_map)
        g.shadow_size = 0 if self.shadow_map is None else self.shadow_map.shape[0]
        g.cam = _camera(self.cam)
        if self.light is not None:
            g.light = _camera(self.light)
        return g


def upload_frame(frame, precision: str = "fp32", device="cuda") -> DeviceFrame:
    """Copy a scenegen.Frame to the device in the storage format of `precision`."""
    ndt = torch.float16 if precision == "fp16" else torch.float32
    depth = torch.from_numpy(frame.depth).to(device)
    normal = torch.from_numpy(frame.normal).to(device=device, dtype=ndt)
    color = torch.from_numpy(frame.color).to(device=device, dtype=torch.float16)
    sm = None
    if frame.shadow_map is not None:
        sm = torch.from_numpy(frame.shadow_map).to(device=device, dtype=torch.float32)  # FP32 in both precisions
    return DeviceFrame(frame.width, frame.height, depth, normal.contiguous(), frame.cam, color.contiguous(), sm,
                       frame.light)


@dataclass
class Levels:
    """Caller-owned per-level mask buffers (mrr_levels) as torch tensors."""
    num_levels: int
    dims: list
    alpha: list
    stencil: list
    worklist: list
    counts: torch.Tensor
    label: torch.Tensor | None

    def struct(self) -> mrr_levels:
        lv = mrr_levels()
        lv.num_levels = self.num_levels
        for i in range(self.num_levels):
            lv.width[i], lv.height[i] = self.dims[i]
            lv.alpha[i] = _ptr(self.alpha[i])
            lv.stencil[i] = _ptr(self.stencil[i])
            lv.worklist[i] = _ptr(self.worklist[i])
        lv.counts = _ptr(self.counts)
        lv.label = _ptr(self.label)
        return lv


def alloc_levels(width: int, height: int, num_levels: int, with_label: bool = True, device="cuda") -> Levels:
    dims = [mrr_level_dims(width, height, i) for i in range(num_levels)]
    alpha = [torch.empty((h, w), dtype=torch.float32, device=device) for (w, h) in dims]
    stencil = [torch.empty((h, w), dtype=torch.uint8, device=device) for (w, h) in dims]
    worklist = [torch.empty((h * w,), dtype=torch.int32, device=device) for (w, h) in dims]
    counts = torch.zeros((MAX_LEVELS,), dtype=torch.int32, device=device)
    label = torch.empty((height, width), dtype=torch.uint8, device=device) if with_label else None
    return Levels(num_levels, dims, alpha, stencil, worklist, counts, label)


def alloc_subimages(ctx: Context, width: int, height: int, device="cuda") -> list:
    dt = torch.float16 if ctx.config.get("precision", "fp32") == "fp16" else torch.float32
    out = []
    full_res = bool(ctx.config.get("sample_levels", 0))   # sample-count levels: [H][W] above level 0
    for i in range(ctx.config["num_levels"]):
        w, h = (width, height) if full_res else mrr_level_dims(width, height, i)
        shape = (h, w, 4) if ctx.channels == 4 else (h, w)
        out.append(torch.full(shape, float("nan"), dtype=dt, device=device) if ctx.config["enabled"][i] else None)
    return out


def alloc_output(ctx: Context, width: int, height: int, device="cuda") -> torch.Tensor:
    shape = (height, width, 4) if ctx.channels == 4 else (height, width)
    return torch.empty(shape, dtype=torch.float32, device=device)


def mrr_edges(ctx: Context, frame: DeviceFrame, edges: torch.Tensor, stream=None) -> None:
    g = frame.struct()
    _check(ctx, _lib.mrr_edges(ctx.handle, ctypes.byref(g), _ptr(edges), _stream(stream)))


def mrr_masks(ctx: Context, edges: torch.Tensor, levels: Levels, stream=None) -> None:
    lv = levels.struct()
    _check(ctx, _lib.mrr_masks(ctx.handle, _ptr(edges), ctypes.byref(lv), _stream(stream)))


def mrr_shade_level(ctx: Context, level: int, frame: DeviceFrame, levels: Levels, c: torch.Tensor,
                    stream=None) -> None:
    g, lv = frame.struct(), levels.struct()
    _check(ctx, _lib.mrr_shade_level(ctx.handle, level, ctypes.byref(g), ctypes.byref(lv), _ptr(c),
                                     _stream(stream)))


def mrr_blur_level(ctx: Context, level: int, frame: DeviceFrame, levels: Levels, c: torch.Tensor, b: torch.Tensor,
                   stream=None) -> None:
    g, lv = frame.struct(), levels.struct()
    _check(ctx, _lib.mrr_blur_level(ctx.handle, level, ctypes.byref(g), ctypes.byref(lv), _ptr(c), _ptr(b),
                                    _stream(stream)))


def mrr_shade_levels(ctx: Context, frame: DeviceFrame, levels: Levels, c_list: list, stream=None) -> None:
    g, lv = frame.struct(), levels.struct()
    arr = (_vp * MAX_LEVELS)(*[(_ptr(c) if c is not None else None) for c in c_list])
    _check(ctx, _lib.mrr_shade_levels(ctx.handle, ctypes.byref(g), ctypes.byref(lv), arr, _stream(stream)))


def mrr_autotune(ctx: Context, frame: DeviceFrame, stream=None) -> dict:
    g = frame.struct()
    t = mrr_tuning()
    _check(ctx, _lib.mrr_autotune(ctx.handle, ctypes.byref(g), _stream(stream), ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in mrr_tuning._fields_}


def mrr_masks_static(cfg: dict, edges: torch.Tensor, levels: Levels, stream=None) -> None:
    """The mask stage without a context and without any allocation (see include/mrr.h).

    The C side cannot check what a device pointer refers to, so the edge image is checked
    here: a uint8 (H, W) tensor on the current CUDA device."""
    if (not isinstance(edges, torch.Tensor) or edges.dtype != torch.uint8 or not edges.is_cuda
            or tuple(edges.shape) != (levels.dims[0][1], levels.dims[0][0]) or not edges.is_contiguous()
            or edges.device.index != torch.cuda.current_device()):
        raise ValueError("edges must be a contiguous uint8 (H, W) tensor on the current CUDA device")
    c, keep = make_config(cfg)
    lv = levels.struct()
    st = _lib.mrr_masks_static(ctypes.byref(c), _ptr(edges), ctypes.byref(lv), _stream(stream))
    if st != MRR_OK:
        raise MrrError(st, "mrr_masks_static")


@dataclass
class Batch:
    handle: int

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _lib.mrr_batch_destroy(h)
            except Exception:
                pass
            self.handle = 0


def mrr_batch_create() -> Batch:
    h = _vp()
    st = _lib.mrr_batch_create(ctypes.byref(h))
    if st != MRR_OK:
        raise MrrError(st, "mrr_batch_create")
    return Batch(h.value)


def mrr_batch_destroy(b: Batch) -> None:
    if b.handle:
        _lib.mrr_batch_destroy(b.handle)
        b.handle = 0


def _batch_args(ctxs, frames):
    n = len(ctxs)
    ca = (_vp * n)(*[c.handle for c in ctxs])
    fa = (mrr_gbuffer * n)(*[f.struct() for f in frames])
    return n, ca, fa


def mrr_render_batch(b: Batch, ctxs: list, frames: list, outs: list, stream=None) -> None:
    """Render frames[k] through ctxs[k] into outs[k] with one batched shading launch."""
    n, ca, fa = _batch_args(ctxs, frames)
    oa = (_vp * n)(*[_ptr(o) for o in outs])
    st = _lib.mrr_render_batch(b.handle, ca, fa, oa, n, _stream(stream))
    if st != MRR_OK:
        raise MrrError(st, "mrr_render_batch: " + _lib.mrr_batch_last_error(b.handle).decode())


def mrr_batch_autotune(b: Batch, ctxs: list, frames: list, stream=None) -> dict:
    n, ca, fa = _batch_args(ctxs, frames)
    t = mrr_batch_tuning()
    st = _lib.mrr_batch_autotune(b.handle, ca, fa, n, _stream(stream), ctypes.byref(t))
    if st != MRR_OK:
        raise MrrError(st, "mrr_batch_autotune: " + _lib.mrr_batch_last_error(b.handle).decode())
    return {k: getattr(t, k) for k, _ in mrr_batch_tuning._fields_}


@dataclass
class Server:
    handle: int
    _keep: list = field(default_factory=list)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _lib.mrr_server_destroy(h)
            except Exception:
                pass
            self.handle = 0


def mrr_server_create(effect_cfgs: dict, slots: int = 4, hbm_reserve: int = 0, max_queue: int = 0,
                      mock_device_us: int = 0, per_effect: int = 0, direct_launches: bool = False) -> Server:
    """effect_cfgs: {'ssao': cfg, 'ssm': cfg, 'ssgi': cfg} (any subset)."""
    sc = mrr_server_config()
    keep = []
    for name, cfg in effect_cfgs.items():
        c, k = make_config(cfg)
        keep.append(k)
        e = EFFECTS[name]
        sc.effect_cfg[e] = c
        sc.effect_enabled[e] = 1
    sc.slots, sc.hbm_reserve, sc.max_queue, sc.mock_device_us = slots, hbm_reserve, max_queue, mock_device_us
    sc.per_effect, sc.direct_launches = per_effect, int(direct_launches)
    h = _vp()
    st = _lib.mrr_server_create(ctypes.byref(sc), ctypes.byref(h))
    if st != MRR_OK:
        raise MrrError(st, "mrr_server_create")
    return Server(h.value)


def mrr_server_destroy(s: Server) -> None:
    if s.handle:
        _lib.mrr_server_destroy(s.handle)
        s.handle = 0


def mrr_server_slots(s: Server) -> int:
    return _lib.mrr_server_slots(s.handle)


def mrr_submit(s: Server, effect: str, frame=None, out: torch.Tensor | None = None) -> int:
    """Queue a request (frame: DeviceFrame or, in mock mode, (width, height)); returns its ticket."""
    r = mrr_request()
    r.effect = EFFECTS[effect]
    if isinstance(frame, DeviceFrame):
        r.frame = frame.struct()
    elif frame is not None:
        r.frame.width, r.frame.height = frame
    r.out_dev = _ptr(out) if out is not None else None
    t = ctypes.c_uint64()
    st = _lib.mrr_submit(s.handle, ctypes.byref(r), ctypes.byref(t))
    if st != MRR_OK:
        raise MrrError(st, "mrr_submit")
    return t.value


def mrr_poll(s: Server, ticket: int):
    done, res = ctypes.c_int(), ctypes.c_int()
    st = _lib.mrr_poll(s.handle, ticket, ctypes.byref(done), ctypes.byref(res))
    if st != MRR_OK:
        raise MrrError(st, "mrr_poll")
    return bool(done.value), res.value


def mrr_wait(s: Server, ticket: int, timeout_ns: int = -1) -> int:
    """Returns the request's status, or MRR_ETIMEDOUT."""
    return _lib.mrr_wait(s.handle, ticket, timeout_ns)


def mrr_request_info(s: Server, ticket: int) -> dict:
    i = mrr_request_info_t()
    st = _lib.mrr_request_info(s.handle, ticket, ctypes.byref(i))
    if st != MRR_OK:
        raise MrrError(st, "mrr_request_info")
    return {k: getattr(i, k) for k, _ in mrr_request_info_t._fields_}


def mrr_server_stats(s: Server) -> dict:
    """Scheduler counters: batches, completed requests, batch graphs instantiated / updated."""
    o = mrr_server_stats_t()
    st = _lib.mrr_server_stats(s.handle, ctypes.byref(o))
    if st != MRR_OK:
        raise MrrError(st, "mrr_server_stats")
    return {k: getattr(o, k) for k, _ in mrr_server_stats_t._fields_}


def mrr_release(s: Server, ticket: int) -> None:
    """Forget a completed request's record (MrrError for an unknown or unfinished ticket)."""
    st = _lib.mrr_release(s.handle, ticket)
    if st != MRR_OK:
        raise MrrError(st, "mrr_release")


def mrr_kernel_launches() -> int:
    return int(_lib.mrr_kernel_launches())


def mrr_check_reciprocal(first_bits: int, last_bits: int) -> int:
    """Mismatches of the kernels' reciprocal against IEEE division over a range of floats."""
    n = ctypes.c_uint64(0)
    _check(None, _lib.mrr_check_reciprocal(first_bits, last_bits, ctypes.byref(n)))
    return int(n.value)


def mrr_check_wait_timeout(ctx: Context) -> int:
    f = ctypes.c_uint32(0)
    _check(ctx, _lib.mrr_check_wait_timeout(ctx.handle, ctypes.byref(f)))
    return int(f.value)


def mrr_fault_flags(ctx: Context, clear: bool = False) -> int:
    """Device fault bits of the context (0: no tile load has stalled)."""
    v = ctypes.c_uint32(0)
    _check(ctx, _lib.mrr_fault_flags(ctx.handle, ctypes.byref(v), int(clear)))
    return int(v.value)


def mrr_upsample_merge(ctx: Context, levels: Levels, c_list: list, out: torch.Tensor, stream=None) -> None:
    lv = levels.struct()
    arr = (_vp * MAX_LEVELS)(*[(_ptr(c) if c is not None else None) for c in c_list])
    _check(ctx, _lib.mrr_upsample_merge(ctx.handle, ctypes.byref(lv), arr, _ptr(out), _stream(stream)))


def mrr_upsample_merge_bilateral(ctx: Context, frame: DeviceFrame, levels: Levels, c_list: list,
                                 out: torch.Tensor, stream=None) -> None:
    g, lv = frame.struct(), levels.struct()
    arr = (_vp * MAX_LEVELS)(*[(_ptr(c) if c is not None else None) for c in c_list])
    _check(ctx, _lib.mrr_upsample_merge_bilateral(ctx.handle, ctypes.byref(g), ctypes.byref(lv), arr, _ptr(out),
                                                  _stream(stream)))


def mrr_render(ctx: Context, frame: DeviceFrame, out: torch.Tensor, stream=None) -> None:
    g = frame.struct()
    _check(ctx, _lib.mrr_render(ctx.handle, ctypes.byref(g), _ptr(out), _stream(stream)))


def mrr_render_full(ctx: Context, frame: DeviceFrame, out: torch.Tensor, stream=None) -> None:
    g = frame.struct()
    _check(ctx, _lib.mrr_render_full(ctx.handle, ctypes.byref(g), _ptr(out), _stream(stream)))


def mrr_trace_shading(ctx: Context, begin=None, end=None) -> None:
    """Record two torch.cuda.Event (enable_timing=True) around the frame path's shading
    launch in every following mrr_render (which then runs without its CUDA graph); no
    events end tracing.  The events must outlive the traced renders."""
    if (begin is None) != (end is None):
        raise ValueError("mrr_trace_shading: both events or neither")
    if begin is None:
        _check(ctx, _lib.mrr_trace_shading(ctx.handle, None, None))
        return
    for ev in (begin, end):
        if not ev.cuda_event:
            ev.record()  # torch creates the underlying event at its first record
    _check(ctx, _lib.mrr_trace_shading(ctx.handle, _vp(begin.cuda_event), _vp(end.cuda_event)))


@dataclass
class HostFrame:
    """A G-buffer in (pinned) host memory, for mrr_render_host."""
    width: int
    height: int
    depth: torch.Tensor
    normal: torch.Tensor
    cam: object
    color: torch.Tensor | None = None
    shadow_map: torch.Tensor | None = None
    light: object = None

    def struct(self) -> mrr_gbuffer:
        g = mrr_gbuffer()
        g.width, g.height = self.width, self.height
        g.depth = self.depth.data_ptr()
        g.normal = self.normal.data_ptr()
        g.color = None if self.color is None else self.color.data_ptr()
        g.shadow_map = None if self.shadow_map is None else self.shadow_map.data_ptr()
        g.shadow_size = 0 if self.shadow_map is None else self.shadow_map.shape[0]
        g.cam = _camera(self.cam)
        if self.light is not None:
            g.light = _camera(self.light)
        return g


def pin_frame(frame, precision: str = "fp32") -> HostFrame:
    ndt = torch.float16 if precision == "fp16" else torch.float32
    pin = lambda a, dt=None: (torch.from_numpy(a) if dt is None else torch.from_numpy(a).to(dt)).contiguous().pin_memory()
    sm = None if frame.shadow_map is None else pin(frame.shadow_map, torch.float32)
    return HostFrame(frame.width, frame.height, pin(frame.depth), pin(frame.normal, ndt), frame.cam,
                     pin(frame.color, torch.float16), sm, frame.light)


def mrr_render_host(ctx: Context, frame: HostFrame, out_host: torch.Tensor, stream=None) -> None:
    g = frame.struct()
    _check(ctx, _lib.mrr_render_host(ctx.handle, ctypes.byref(g), out_host.data_ptr(), _stream(stream)))


# Table 1 of the paper: (sigma_i^2, w_i) of sub-images 1..4 (full, 1/2, 1/4, 1/8 resolution)
# per effect; SSGI does not use the second sub-image (Sec. 4).
TABLE1 = {
    "ssao": [(0.924, 100.0), (1.848, 50.0), (3.696, 20.0), (0.0, 1.0)],
    "ssm": [(0.924, 1000.0), (1.848, 1000.0), (3.696, 1000.0), (0.0, 1.0)],
    "ssgi": [(0.924, 1000.0), None, (0.924, 100.0), (0.0, 1.0)],
}


def mrr_render_host_async(ctx: Context, frame: HostFrame, out_host: torch.Tensor) -> None:
    g = frame.struct()
    _check(ctx, _lib.mrr_render_host_async(ctx.handle, ctypes.byref(g), out_host.data_ptr()))


def mrr_render_host_wait(ctx: Context) -> None:
    _check(ctx, _lib.mrr_render_host_wait(ctx.handle))


def default_config(effect: str, num_levels: int, max_width: int, max_height: int, **kw) -> dict:
    """A configuration dict with Table 1's variances and weights (with three levels the
    coarsest row is used for the third) and this library's defaults for the rest."""
    rows = TABLE1[effect]
    if num_levels == 3:
        rows = [rows[0], rows[1], rows[3]]
    sigma2, weight, enabled = [0.0] * 4, [0.0] * 4, [0] * 4
    for i, row in enumerate(rows[:num_levels]):
        if row is not None:
            sigma2[i], weight[i] = row
            enabled[i] = 1
    cfg = dict(effect=effect, precision="fp32", num_levels=num_levels, sigma2=sigma2, weight=weight,
               enabled=enabled, depth_rel=0.05, normal_cos=0.9, force_level0=0, radius=0.5, ao_bias=0.0125,
               gi_min_dist2=0.01, light_size=0.5, shadow_bias=0.03, max_width=max_width, max_height=max_height,
               blur=[0, 0, 0, 0], blur_depth_rel=0.05, merge_mode=0, sample_levels=0, pyramid_gathers=0,
               disjoint=0)
    cfg.update(kw)
    return cfg
