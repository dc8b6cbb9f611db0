"""Benchmark of the multi-resolution rendering path (arXiv 1906.04576) on one GB300.

One step = one frame through the whole method (edges -> masks -> work lists ->
sub-images -> Eq. (1) blend) via mrr_render, with the G-buffer resident in HBM.
The metric is full-resolution-equivalent Mpixels/s (W*H per frame time), reported
beside the plain full-resolution kernel (mrr_render_full) on the same frame, the
RMSE between the two, p50/p99 frame times, the roofline of the dominant kernel
(the work-list shading kernel), an end-to-end figure through mrr_render_host (host
G-buffer in, host image out), and the CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

N > 1 (under torchrun): independent replicas, each rank renders its own seeded frames;
value = all ranks' pixels / the slowest rank's time ("replicas only": the method has
no cross-GPU exchange).  L2 is flushed (a 256 MiB write) before every timed step,
outside the timed events.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "full-res-equiv Mpix/s multires vs plain full-res at RMSE<=1e-2; p50/p99 frame ms"
FLUSH_BYTES = 256 << 20
SCENES = 24  # seeded scenes per configuration, in rotation over the timed steps


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def pct(vals, q):
    s = sorted(vals)
    if not s:
        return float("nan")
    k = (len(s) - 1) * q
    lo, hi = math.floor(k), math.ceil(k)
    return s[lo] + (s[hi] - s[lo]) * (k - lo)


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_rejected(clocks):
    """A timed region whose clock record shows a hardware or thermal slowdown, or SM clocks
    well below their maximum with no reason reported (a clock lock left behind), is not a
    valid measurement and is taken again once; sw_power_cap alone is kept and noted."""
    reasons = set(clocks.get("reasons") or [])
    if reasons & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        return True
    sm, smax = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    return bool(sm and smax and not reasons and sm < 0.9 * smax)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


SHADE_SOURCES = ["paper_1906_04576_gb300/csrc/k_shade.cu", "paper_1906_04576_gb300/csrc/shade_common.cuh",
                 "paper_1906_04576_gb300/csrc/mrr_internal.cuh"]


def shade_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in SHADE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    """DRAM bytes per launch of the work-list kernel from a committed ncu capture
    (profiles/traffic_<workload>.json), only while the kernel sources are unchanged."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d["dram_bytes_per_launch"] if d.get("sources_sha") == shade_sources_sha() else None


def algorithmic_bytes(cfg, n_nonsky, n_sky):
    """Bytes the shading kernel must move per launch by definition of the effect:
    per non-sky texel its depth + normal, every sample's gathers and the store; per sky
    texel its depth and the store."""
    half = cfg.get("precision", "fp32") == "fp16"
    nb = 8 if half else 16
    eff = cfg["effect"]
    if eff == "ssao":
        per, store = 4 + nb + cfg["samples"] * 4, (2 if half else 4)
    elif eff == "ssgi":
        per, store = 4 + nb + cfg["samples"] * (4 + nb + 8), (8 if half else 16)
    else:
        # the shadow map stays FP32 in both storage precisions
        per, store = 4 + (cfg["blocker_samples"] + cfg["pcf_samples"]) * 4, (2 if half else 4)
    return n_nonsky * (per + store) + n_sky * (4 + store)


def effect_config(mrr, sg, spec, W, H, precision):
    eff = spec["effect"]
    kw = {}
    if eff in ("ssao", "ssgi"):
        kw.update(kernel=sg.hemisphere_kernel(spec["samples"]), radius=spec["radius"], samples=spec["samples"])
    else:
        kw.update(blocker_taps=sg.disk_taps(spec["blocker_samples"], sg.BLOCKER_SEED),
                  pcf_taps=sg.disk_taps(spec["pcf_samples"], sg.PCF_SEED),
                  blocker_samples=spec["blocker_samples"], pcf_samples=spec["pcf_samples"])
    if "blur" in spec:
        kw.update(blur=list(spec["blur"]))
    if "merge_mode" in spec:
        kw.update(merge_mode=spec["merge_mode"])
    if "sample_levels" in spec:
        kw.update(sample_levels=spec["sample_levels"])
    if "pyramid_gathers" in spec:
        kw.update(pyramid_gathers=spec["pyramid_gathers"])
    if "disjoint" in spec:
        kw.update(disjoint=spec["disjoint"])
    return mrr.default_config(eff, spec["levels"], W, H, precision=precision, **kw)


def workload_config(mrr, sg, name):
    wl = dict(sg.WORKLOADS[name])
    cfg = effect_config(mrr, sg, wl, wl["width"], wl["height"], wl.get("precision", "fp32"))
    return wl, cfg


def config_of(name, wl, rank, world):
    """The workload's config dict, the same for both arms (the library and the oracle)."""
    W, H = wl["width"], wl["height"]
    return {"workload": name, "width": W, "height": H, "effect": wl["effect"],
            "samples": wl.get("samples"), "levels": wl["levels"], "precision": wl.get("precision", "fp32"),
            "blur": list(wl.get("blur", [0, 0, 0, 0])),
            "merge": {0: "direct (Sec. 4.2)", 1: "step-wise (Sec. 3.3)",
                      2: "direct, bilateral taps (Sec. 3.3)"}[wl.get("merge_mode", 0)],
            "levels_kind": "sample-count (Sec. 6)" if wl.get("sample_levels", 0) else "resolution",
            "pyramid_gathers": bool(wl.get("pyramid_gathers", 0)),
            "decomposition": "disjoint tiles (Sec. 3.1 ablation)" if wl.get("disjoint", 0) else "inclusive nesting",
            "scene": f"{wl['n_boxes']} boxes + {wl['n_spheres']} spheres, {SCENES} seeded scenes "
                     f"(seeds {SCENES * rank}..{SCENES * rank + SCENES - 1}) in rotation, one per step",
            "l2": "GPU arm: L2 flushed (256 MiB write) before every timed step, outside the events; "
                  "every step's G-buffer is larger than any cache",
            "parallelism": f"replicas x{world}"}


def make_frame(sg, wl, seed):
    return sg.gbuffer(seed, wl["width"], wl["height"], wl["n_boxes"], wl["n_spheres"],
                      shadow_size=wl.get("shadow_size", 0))


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the oracle timing."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_config(orc, sg, wl):
    """The oracle's configuration of a workload (the same parameters the library gets)."""
    eff = wl["effect"]
    kw = {}
    if eff in ("ssao", "ssgi"):
        kw.update(kernel=sg.hemisphere_kernel(wl["samples"]), samples=wl["samples"], radius=wl["radius"])
    else:
        kw.update(blocker_taps=sg.disk_taps(wl["blocker_samples"], sg.BLOCKER_SEED),
                  pcf_taps=sg.disk_taps(wl["pcf_samples"], sg.PCF_SEED))
    if "blur" in wl:
        kw.update(blur=list(wl["blur"]))
    if "merge_mode" in wl:
        kw.update(merge_mode=wl["merge_mode"])
    if "sample_levels" in wl:
        kw.update(sample_levels=wl["sample_levels"])
    if "pyramid_gathers" in wl:
        kw.update(pyramid_gathers=wl["pyramid_gathers"])
    if "disjoint" in wl:
        kw.update(disjoint=wl["disjoint"])
    return orc.default_config(eff, wl["levels"], **kw)


def cpu_oracle_sample(sg, wl, name, budget_s=10.0, max_frames=2000):
    """The oracle, as it stands, rendering whole frames of the workload on the host cores
    until about budget_s seconds of CPU work have been spent."""
    import oracle as orc
    fr = make_frame(sg, wl, 0)
    cfg = oracle_config(orc, sg, wl)
    orc.render(fr, cfg, "f32")   # warm-up (page-in, thread pool)
    n, t0 = 0, time.perf_counter()
    times = []
    while n < max_frames and (time.perf_counter() - t0) < budget_s or n < 2:
        t = time.perf_counter()
        orc.render(fr, cfg, "f32")
        times.append(time.perf_counter() - t)
        n += 1
    total = sum(times)
    cores = orc.num_threads()
    # one frame on a single host thread, beside the all-cores figure
    orc.set_threads(1)
    t = time.perf_counter()
    orc.render(fr, cfg, "f32")
    t1 = time.perf_counter() - t
    orc.set_threads(cores)
    return {"value": round(n * wl["width"] * wl["height"] / total / 1e6, 4), "unit": "Mpix/s",
            "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{n} whole {wl['width']}x{wl['height']} frames of {name} (float oracle, OpenMP over rows)",
            "seconds": round(total, 3),
            "single_thread": {"value": round(wl["width"] * wl["height"] / t1 / 1e6, 4), "unit": "Mpix/s",
                              "sample": "one frame on one host thread"}}


def run_reference(args):
    """The oracle as the reference arm: same workload, metric and unit, on host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import scenegen as sg
    import oracle as orc
    sg.build()
    orc.build()
    wl = dict(sg.WORKLOADS[args.workload])
    if wl["effect"] == "mix" or "batch_with" in wl:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle renders single frames; the "
                          "serving mix and batched workloads have no oracle arm"}), flush=True)
        return 0
    cfg = oracle_config(orc, sg, wl)
    # the GPU arm's scenes (seeds 0..SCENES-1), ray-cast once, one per step in rotation
    frames = [make_frame(sg, wl, k) for k in range(SCENES)]
    for _ in range(max(1, min(args.warmup, 3))):
        orc.render(frames[0], cfg, "f32")
    t = time.perf_counter()
    orc.render(frames[1], cfg, "f32")
    est = time.perf_counter() - t
    budget = 150.0
    steps = args.steps if args.steps * est <= budget else max(3, int(budget / est))
    times = []
    for k in range(steps):
        t = time.perf_counter()
        orc.render(frames[k % SCENES], cfg, "f32")
        times.append((time.perf_counter() - t) * 1e3)
    W, H = wl["width"], wl["height"]
    total_s = sum(times) / 1e3
    value = steps * W * H / total_s / 1e6
    sample = f"{steps} whole {W}x{H} frames, scenes in rotation (float oracle, OpenMP over rows)"
    if steps != args.steps:
        sample += f"; {args.steps} requested, capped at {budget:.0f} s of CPU work"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpix/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(total_s * 1e3 / steps, 4),
            "p50_ms": round(pct(times, 0.5), 4), "p99_ms": round(pct(times, 0.99), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_of(args.workload, wl, rank, world),
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpix/s", "cores": orc.num_threads(),
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, mrr, sg, wl, rank, world, dist):
    """The serving mix: seeded Poisson arrivals of frame requests, uniform over
    resolutions x effects, submitted to one server as they arrive; throughput
    (full-resolution-equivalent Mpix/s over the whole run) and p50/p99 latency
    (completion - arrival).  G-buffers come from a pool of seeded scenes made before
    the timed run and resident on the device."""
    import numpy as np
    import torch
    Wm, Hm = max(r[0] for r in wl["resolutions"]), max(r[1] for r in wl["resolutions"])
    specs = wl["effects"]
    names = [e["effect"] for e in specs]
    cfgs = {e["effect"]: effect_config(mrr, sg, e, Wm, Hm, e["precision"]) for e in specs}
    srv = mrr.mrr_server_create(cfgs, slots=wl["slots"], hbm_reserve=8 << 30, per_effect=wl.get("per_effect", 2))
    slots = mrr.mrr_server_slots(srv)
    # resident G-buffer pool: scenes_per_resolution seeded scenes per resolution
    pool = {}
    for ri, (W, H) in enumerate(wl["resolutions"]):
        for k in range(wl["scenes_per_resolution"]):
            seed = 1000 * rank + 10 * ri + k
            fr = sg.gbuffer(seed, W, H, wl["n_boxes"], wl["n_spheres"], shadow_size=2048)
            pool[(ri, k, "fp32")] = mrr.upload_frame(fr, "fp32")
            pool[(ri, k, "fp16")] = mrr.upload_frame(fr, "fp16")
    prec = {e["effect"]: e["precision"] for e in specs}
    n_req = wl["requests"]
    gaps, pick = sg.poisson_stream(0xA11 + rank, n_req, wl["rate"], len(wl["resolutions"]) * len(names))
    scene_pick = np.arange(n_req) % wl["scenes_per_resolution"]
    # every request gets an output buffer of its own (kept until it completes), and
    # consecutive requests of one resolution read different G-buffers: the batches' graphs
    # are keyed on topology, never on pointers
    def fresh_out(ri, e):
        W, H = wl["resolutions"][ri]
        return torch.empty((H, W, 4) if e == "ssgi" else (H, W), dtype=torch.float32, device="cuda")
    # warm-up: one request of every kind
    for ri in range(len(wl["resolutions"])):
        for e in names:
            t = mrr.mrr_submit(srv, e, pool[(ri, 0, prec[e])], fresh_out(ri, e))
            mrr.mrr_wait(srv, t, -1)
    torch.cuda.synchronize()
    stats0 = mrr.mrr_server_stats(srv)
    if dist is not None:
        dist.barrier()
    tickets, pixels, live = [], 0, {}
    t_start = time.perf_counter()
    arrival = t_start
    l0 = mrr.mrr_kernel_launches()
    for i in range(n_req):
        arrival += gaps[i]
        while time.perf_counter() < arrival:
            pass
        ri, ei = divmod(int(pick[i]), len(names))
        e = names[ei]
        W, H = wl["resolutions"][ri]
        out = fresh_out(ri, e)
        t = mrr.mrr_submit(srv, e, pool[(ri, int(scene_pick[i]), prec[e])], out)
        live[t] = out
        tickets.append(t)
        pixels += W * H
        # outputs of finished requests go back to the allocator
        if i % 64 == 63:
            for tk in [tk for tk in live if mrr.mrr_poll(srv, tk)[0]]:
                del live[tk]
    for t in tickets:
        mrr.mrr_wait(srv, t, -1)
    t_end = time.perf_counter()
    launches = mrr.mrr_kernel_launches() - l0
    stats1 = mrr.mrr_server_stats(srv)
    live.clear()
    info = [mrr.mrr_request_info(srv, t) for t in tickets]
    lat = [(i["done_ns"] - i["submit_ns"]) * 1e-6 for i in info]
    qwait = [(i["start_ns"] - i["submit_ns"]) * 1e-6 for i in info]
    span = max(i["done_ns"] for i in info) - min(i["submit_ns"] for i in info)
    wall = max_reduce(dist, span * 1e-9)
    offered_s = float(np.sum(gaps))
    mrr.mrr_server_destroy(srv)
    if rank == 0:
        value = world * pixels / wall / 1e6
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Mpix/s", "n_gpus": world, "steps": n_req,
            "warmup": len(wl["resolutions"]) * len(names), "ms_per_step": round(wall * 1e3 / n_req, 5),
            "p50_ms": round(pct(lat, 0.5), 4), "p99_ms": round(pct(lat, 0.99), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (SSGI f16-storage)",
            "data": "synthetic", "config": {
                "workload": args.workload, "arrivals": f"Poisson {wl['rate']:.0f}/s, {n_req} requests",
                "mix": "uniform over " + ", ".join(f"{w}x{h}" for w, h in wl["resolutions"]) + " x " + ", ".join(names),
                "slots": slots, "per_effect": wl.get("per_effect", 2),
                "scenes": f"{wl['scenes_per_resolution']} seeded scenes per resolution, resident, in rotation; "
                          "a new output buffer per request",
                "l2": "not flushed: a live request stream", "parallelism": f"replicas x{world}"},
            "offered_mpix_s": round(pixels / offered_s / 1e6, 3),
            "sustained": bool(wall <= offered_s * 1.05),
            "queue_wait_p50_ms": round(pct(qwait, 0.5), 4), "queue_wait_p99_ms": round(pct(qwait, 0.99), 4),
            "device_ms_p50": round(pct([i["device_ms"] for i in info], 0.5), 4),
            "batches": int(stats1["batches"] - stats0["batches"]),
            "graph_instantiations": int(stats1["graph_instantiations"] - stats0["graph_instantiations"]),
            "graph_updates": int(stats1["graph_updates"] - stats0["graph_updates"]),
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    return 0


def max_reduce(dist, x, device="cuda"):
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(world, steps, pixels_per_step, slowest_rank_ms):
    """Throughput of the whole job: every rank's pixels over the slowest rank's time."""
    return world * steps * pixels_per_step / (slowest_rank_ms * 1e-3) / 1e6


def run_batch(args, mrr, sg, wl, cfg, rank, world, dist):
    """One step = both effects of the workload on one frame through mrr_render_batch
    (one batched shading launch), against the two plain full-resolution kernels."""
    import torch
    W, H = wl["width"], wl["height"]
    prec = cfg["precision"]
    cfg2 = effect_config(mrr, sg, wl["batch_with"], W, H, prec)
    frames = [make_frame(sg, wl, SCENES * rank + k) for k in range(SCENES)]
    ctxs = [mrr.mrr_create(cfg), mrr.mrr_create(cfg2)]
    scenes = [mrr.upload_frame(f, prec) for f in frames]
    dev = mrr.upload_frame(frames[0], prec)

    def load_scene(k):
        src = scenes[k % SCENES]
        dev.depth.copy_(src.depth)
        dev.normal.copy_(src.normal)
        dev.color.copy_(src.color)

    outs = [mrr.alloc_output(c, W, H) for c in ctxs]
    fulls = [mrr.alloc_output(c, W, H) for c in ctxs]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    b = mrr.mrr_batch_create()
    tune = None if args.no_tune else mrr.mrr_batch_autotune(b, ctxs, [dev, dev], stream)
    step = lambda: mrr.mrr_render_batch(b, ctxs, [dev, dev], outs, stream)

    def step_full():
        for c, o in zip(ctxs, fulls):
            mrr.mrr_render_full(c, dev, o, stream)

    for _ in range(args.warmup):
        step()
        step_full()
    torch.cuda.synchronize()

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        for k, (s_, e_) in enumerate(ev):
            load_scene(k)
            flush.zero_()
            s_.record(stream)
            fn()
            e_.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        return [s_.elapsed_time(e_) for s_, e_ in ev]

    def max_over_ranks(x):
        return max_reduce(dist, x)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    first_clocks = None
    for attempt in range(2):
        sampler = ClockSampler(vis.split(",")[int(os.environ.get("LOCAL_RANK", "0"))].strip() if vis
                               else torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
        l0 = mrr.mrr_kernel_launches()
        t_b = timed(step, args.steps)
        launches = mrr.mrr_kernel_launches() - l0
        t_f = timed(step_full, args.steps)
        clocks = sampler.stop()
        # a rejected clock record on any rank: the whole timed region once more
        if attempt == 1 or max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0) == 0.0:
            break
        first_clocks = clocks

    # quality gate per effect: the worst scene's RMSE (and the mean) over the 24 scenes
    per_scene = [[], []]
    for k in range(SCENES):
        load_scene(k)
        step()
        step_full()
        torch.cuda.synchronize()
        for j, (o, f_) in enumerate(zip(outs, fulls)):
            d = (o - f_)[..., :3] if o.dim() == 3 else (o - f_)
            per_scene[j].append(float(torch.sqrt(torch.mean(d.double() ** 2)).item()))
    rmse = [max(v) for v in per_scene]
    rmse_mean = [round(statistics.mean(v), 6) for v in per_scene]
    sb, sf = max_over_ranks(sum(t_b)), max_over_ranks(sum(t_f))
    value = whole_job_mpix_s(world, args.steps, 2 * W * H, sb)
    fvalue = whole_job_mpix_s(world, args.steps, 2 * W * H, sf)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sb / args.steps, 5), "p50_ms": round(pct(t_b, 0.5), 5),
            "p99_ms": round(pct(t_b, 0.99), 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16-storage/f32" if prec == "fp16" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "width": W, "height": H,
                       "effects": [cfg["effect"], cfg2["effect"]], "samples": [cfg.get("samples"), cfg2.get("samples")],
                       "precision": prec, "batch": "both effects of one frame in one persistent shading launch",
                       "scene": f"{wl['n_boxes']} boxes + {wl['n_spheres']} spheres, {SCENES} seeded scenes "
                                f"(seeds {SCENES * rank}..{SCENES * rank + SCENES - 1}) in rotation, one per step",
                       "l2": "flushed (256 MiB write) before every timed step, outside the events",
                       "parallelism": f"replicas x{world}"},
            "full_res": {"value": round(fvalue, 3), "unit": "Mpix/s", "p50_ms": round(pct(t_f, 0.5), 5),
                         "p99_ms": round(pct(t_f, 0.99), 5)},
            "speedup_vs_full_res": round(value / fvalue, 4), "rmse_vs_full_res": rmse, "rmse_mean": rmse_mean,
            "gpu_launches": int(launches), "tuning": tune, "clocks": clocks,
            **({"remeasured": {"first_clocks": first_clocks}} if first_clocks is not None else {}),
        }
        print(json.dumps(line), flush=True)
    mrr.mrr_batch_destroy(b)
    for c in ctxs:
        mrr.mrr_destroy(c)
    return 0


def main():
    global SCENES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="ssao64_4k")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip mrr_autotune (library defaults)")
    ap.add_argument("--scenes", type=int, default=SCENES,
                    help="seeded scenes in rotation (fewer keep a profiler capture's device memory small)")
    ap.add_argument("--rate", type=float, default=None,
                    help="serving mix only: mean request rate per second (default: the workload's)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    SCENES = max(1, args.scenes)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    import paper_1906_04576_gb300 as mrr
    import scenegen as sg

    if sg.WORKLOADS[args.workload]["effect"] == "mix":
        wl = dict(sg.WORKLOADS[args.workload])
        if args.rate:
            wl["rate"] = args.rate
        return run_serve(args, mrr, sg, wl, rank, world, dist)
    wl, cfg = workload_config(mrr, sg, args.workload)
    W, H = wl["width"], wl["height"]
    prec = cfg["precision"]
    if "batch_with" in wl:
        return run_batch(args, mrr, sg, wl, cfg, rank, world, dist)
    # SCENES seeded scenes (seeds SCENES*rank .. +SCENES-1), all resident; before each timed
    # step the next one is copied into the frame buffers the renders read (outside the
    # events), so every step is a different scene while the captured launches stay valid
    frames = [make_frame(sg, wl, SCENES * rank + k) for k in range(SCENES)]
    fr = frames[0]
    ctx = mrr.mrr_create(cfg)
    scenes = [mrr.upload_frame(f, prec) for f in frames]
    dev = mrr.upload_frame(fr, prec)
    out = mrr.alloc_output(ctx, W, H)
    full = mrr.alloc_output(ctx, W, H)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def load_scene(k):
        src = scenes[k % SCENES]
        dev.depth.copy_(src.depth)
        dev.normal.copy_(src.normal)
        dev.color.copy_(src.color)
        if dev.shadow_map is not None:
            dev.shadow_map.copy_(src.shadow_map)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return max_reduce(dist, x)

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        for k, (s, e) in enumerate(ev):
            load_scene(k)
            flush.zero_()
            s.record(stream)
            fn()
            e.record(stream)
        barrier()
        return [s.elapsed_time(e) for s, e in ev]

    tuning = None if args.no_tune else mrr.mrr_autotune(ctx, dev, stream)
    render = lambda: mrr.mrr_render(ctx, dev, out, stream)
    render_full = lambda: mrr.mrr_render_full(ctx, dev, full, stream)
    for _ in range(args.warmup):
        render()
        render_full()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    first_clocks = None
    for attempt in range(2):
        sampler = ClockSampler(vis.split(",")[local].strip() if vis else torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
        l0 = mrr.mrr_kernel_launches()
        t_multi = timed(render, args.steps)
        launches = mrr.mrr_kernel_launches() - l0
        t_full = timed(render_full, args.steps)

        # dominant kernel: the frame path's work-list shading launch, timed inside whole
        # frames of scene 0 (L2 flushed before each, as in the timed loop) with CUDA events
        # that the library records on the launching stream around that launch
        # (mrr_trace_shading)
        load_scene(0)
        edges = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        levels = mrr.alloc_levels(W, H, cfg["num_levels"], with_label=False)
        mrr.mrr_edges(ctx, dev, edges, stream)
        mrr.mrr_masks(ctx, edges, levels, stream)
        tb, te = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        mrr.mrr_trace_shading(ctx, tb, te)
        k_times = []
        for _ in range(max(10, args.steps // 4)):
            flush.zero_()
            mrr.mrr_render(ctx, dev, out, stream)
            stream.synchronize()
            k_times.append(tb.elapsed_time(te))
        mrr.mrr_trace_shading(ctx)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        # a rejected clock record on any rank: the whole timed region once more
        if attempt == 1 or max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0) == 0.0:
            break
        first_clocks = clocks
    k_ms = statistics.mean(k_times)

    # e2e: host G-buffer in, host image out, through the public host API: the pipelined
    # mrr_render_host_async (each step's upload overlapping the previous step's rendering
    # and download), and the synchronous mrr_render_host beside it
    host = mrr.pin_frame(fr, prec)
    out_h = torch.empty(tuple(out.shape), dtype=torch.float32).pin_memory()
    e2e_steps = max(10, args.steps // 2)
    for _ in range(3):
        mrr.mrr_render_host_async(ctx, host, out_h)
    mrr.mrr_render_host_wait(ctx)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mrr.mrr_render_host_async(ctx, host, out_h)
    mrr.mrr_render_host_wait(ctx)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    for _ in range(3):
        mrr.mrr_render_host(ctx, host, out_h, stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mrr.mrr_render_host(ctx, host, out_h, stream)
    barrier()
    e2e_sync_s = max_over_ranks(time.perf_counter() - t0)
    h2d = host.depth.numel() * 4 + host.normal.numel() * host.normal.element_size()
    if cfg["effect"] == "ssgi":
        h2d += host.color.numel() * 2
    if host.shadow_map is not None:
        h2d += host.shadow_map.numel() * host.shadow_map.element_size()
    d2h = out_h.numel() * 4

    # quality gate: RMSE of the multi-resolution image against full-resolution shading,
    # every scene (the gate is the worst one); texels shaded per scene
    rmses, rmses_ns, shaded, dead, rmses_black = [], [], [], [], []
    for k in range(SCENES):
        load_scene(k)
        mrr.mrr_render(ctx, dev, out, stream)
        mrr.mrr_render_full(ctx, dev, full, stream)
        mrr.mrr_edges(ctx, dev, edges, stream)
        mrr.mrr_masks(ctx, edges, levels, stream)
        torch.cuda.synchronize()
        diff = (out - full)[..., :3] if out.dim() == 3 else (out - full)
        nonsky = dev.depth < fr.cam.far
        if cfg.get("disjoint", 0):
            # the ablation's dead pixels are undefined (NaN): the RMSE is over the defined
            # pixels, beside their count and the RMSE with dead pixels drawn black
            nanmask = torch.isnan(out)
            black = torch.where(nanmask, torch.zeros_like(out), out)
            db = (black - full)[..., :3] if out.dim() == 3 else (black - full)
            rmses_black.append(float(torch.sqrt(torch.mean(db.double() ** 2)).item()))
            defined = ~(nanmask[..., 0] if out.dim() == 3 else nanmask)
            dead.append(int((~defined).sum().item()))
            diff = diff[defined]
            nonsky = nonsky[defined]
        rmses.append(float(torch.sqrt(torch.mean(diff.double() ** 2)).item()))
        dns = diff[nonsky] if diff.dim() <= 2 else diff[nonsky.unsqueeze(-1).expand_as(diff)]
        rmses_ns.append(float(torch.sqrt(torch.mean(dns.double() ** 2)).item()) if dns.numel() else 0.0)
        shaded.append(int(levels.counts[: cfg["num_levels"]].sum().item()))
    rmse = max(rmses)
    load_scene(0)
    mrr.mrr_edges(ctx, dev, edges, stream)
    mrr.mrr_masks(ctx, edges, levels, stream)
    torch.cuda.synchronize()

    import numpy as np
    counts = levels.counts.cpu().tolist()
    depth_host = fr.depth
    n_sky = n_all = 0
    alg = 0
    sample_levels = bool(cfg.get("sample_levels", 0))
    for i in range(cfg["num_levels"]):
        if not cfg["enabled"][i] or counts[i] == 0:
            continue
        wlst = levels.worklist[i][: counts[i]].cpu().numpy().view("uint32")
        qy, qx = wlst >> 16, wlst & 0xFFFF
        if sample_levels and i > 0:
            # every pixel of each listed block, with every 2^i-th sample
            dy, dx = np.meshgrid(np.arange(1 << i), np.arange(1 << i), indexing="ij")
            py = ((qy.astype("int64") << i)[:, None] + dy.reshape(1, -1)).reshape(-1)
            px = ((qx.astype("int64") << i)[:, None] + dx.reshape(1, -1)).reshape(-1)
            keep = (py < H) & (px < W)
            sky = int((depth_host[py[keep], px[keep]] >= fr.cam.far).sum())
            npx = int(keep.sum())
            thin = dict(cfg)
            for key in ("samples", "blocker_samples", "pcf_samples"):
                if cfg.get(key):
                    thin[key] = -(-cfg[key] // (1 << i))
            alg += algorithmic_bytes(thin, npx - sky, sky)
            n_sky += sky
            n_all += npx
            continue
        o = 0 if i == 0 else (1 << (i - 1))
        sy = (qy.astype("int64") << i) + o
        sx = (qx.astype("int64") << i) + o
        sy[sy > H - 1] = H - 1
        sx[sx > W - 1] = W - 1
        sky = int((depth_host[sy, sx] >= fr.cam.far).sum())
        alg += algorithmic_bytes(cfg, counts[i] - sky, sky)
        n_sky += sky
        n_all += counts[i]
    peak, peak_kind = measured_peaks()
    achieved = alg / (k_ms * 1e-3) / 1e9

    sum_multi = max_over_ranks(sum(t_multi))
    sum_full = max_over_ranks(sum(t_full))
    value = whole_job_mpix_s(world, args.steps, W * H, sum_multi)
    full_value = whole_job_mpix_s(world, args.steps, W * H, sum_full)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sum_multi / args.steps, 5),
            "p50_ms": round(pct(t_multi, 0.5), 5), "p99_ms": round(pct(t_multi, 0.99), 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16-storage/f32" if prec == "fp16" else "f32", "data": "synthetic",
            "config": config_of(args.workload, wl, rank, world),
            "full_res": {"value": round(full_value, 3), "unit": "Mpix/s", "p50_ms": round(pct(t_full, 0.5), 5),
                         "p99_ms": round(pct(t_full, 0.99), 5)},
            "speedup_vs_full_res": round(value / full_value, 4),
            "rmse_vs_full_res": rmse, "rmse_mean": round(statistics.mean(rmses), 6),
            "rmse_nonsky": round(max(rmses_ns), 6),
            "shaded_texels_mean": round(statistics.mean(shaded), 1),
            "shaded_texels": n_all, "shaded_fraction": round(n_all / (W * H), 5),
            **({"dead_pixels_max": max(dead), "dead_fraction_max": round(max(dead) / (W * H), 6),
                "rmse_dead_black_max": round(max(rmses_black), 6)} if dead else {}),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": measured_traffic(args.workload),
                         "kernel": "shade_levels_kernel" + (" + shade_blocks_kernel" if sample_levels else ""),
                         "kernel_ms": round(k_ms, 5),
                         "algorithmic_bytes": int(alg), "peak_kind": f"{peak_kind} hbm_gbs"},
            "e2e": {"value": round(world * e2e_steps * W * H / e2e_s / 1e6, 3), "unit": "Mpix/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "api": "mrr_render_host_async + mrr_render_host_wait (pinned host buffers; each step's "
                           "upload overlaps the previous step's rendering and download; scene 0)",
                    "sync": {"value": round(world * e2e_steps * W * H / e2e_sync_s / 1e6, 3), "unit": "Mpix/s",
                             "api": "mrr_render_host (copies, rendering and sync inside every call)"}},
            "gpu_launches": int(launches),
            "tuning": tuning,
            "clocks": clocks,
            **({"remeasured": {"first_clocks": first_clocks}} if first_clocks is not None else {}),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_sample(sg, wl, args.workload)
        print(json.dumps(line), flush=True)
    mrr.mrr_destroy(ctx)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
