"""Autotuner for the reconstruction kernels' launch shape.

Picks the tile width (pixels per CTA along a row) and the number of thread
groups splitting the bins by timing candidate plans on the device with CUDA
events, and caches the winner per shape class (GPU, kernel, columns, steps,
bins, output type, geometry precision) in a JSON file.  Every candidate
computes bitwise the same result; only the speed differs.
"""
from __future__ import annotations

import json
import os
import threading

from . import dr

ROWS_CANDIDATES = ((128, 16), (128, 8), (256, 8), (256, 4), (64, 16), (128, 4))
PIXELS_CANDIDATES = ((32, 16), (16, 32), (16, 16), (8, 64), (32, 8), (64, 8), (128, 4), (64, 4))

_lock = threading.Lock()


def cache_path():
    return os.environ.get("DR_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2201_13309_gb300", "tune.json")


def shape_key(gpu, kernel, cols, K, B, out_dtype, geom_precision):
    kb = 1 << max(0, (int(K) - 1).bit_length())       # steps bucket (power of two)
    bb = 1 << max(0, (int(B) - 1).bit_length())       # bins bucket
    return f"{gpu}|{kernel}|W{int(cols)}|K{kb}|B{bb}|{out_dtype}|{geom_precision}"


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(key, value, path=None):
    path = path or cache_path()
    with _lock:
        d = load_cache(path)
        d[key] = value
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def candidates(kernel):
    return ROWS_CANDIDATES if kernel == "rows" else PIXELS_CANDIDATES


def tune(geom, wires, edges, images, out=None, edge="leading", out_dtype="f32",
         geom_precision="fp32", force_pixels=False, reps=8, use_cache=True, stream=None):
    """Best (tile_cols, bin_groups) for this scan shape, timed on ``images``
    (a CUDA tensor [K, rows, cols]).  Returns a dict with the choice, its time
    and every candidate's time."""
    import torch

    probe = dr.Plan(geom, wires, edges, edge=edge, out_dtype=out_dtype,
                    geom_precision=geom_precision, force_pixels=force_pixels)
    info = probe.info()
    gpu = torch.cuda.get_device_name(images.device)
    key = shape_key(gpu, info["kernel"], info["cols"], info["K"], info["B"], out_dtype,
                    geom_precision)
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            return dict(hit, cached=True, key=key)
    if out is None:
        out = probe.empty_output(images.device)
    stream = stream or torch.cuda.current_stream(images.device)
    timings = []
    for tc, bg in candidates(info["kernel"]):
        try:
            plan = dr.Plan(geom, wires, edges, edge=edge, out_dtype=out_dtype,
                           geom_precision=geom_precision, tile_cols=tc, bin_groups=bg,
                           force_pixels=force_pixels)
        except dr.DrError:
            continue
        for _ in range(2):
            plan.reconstruct(images, out, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.reconstruct(images, out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        timings.append({"tile_cols": tc, "bin_groups": bg, "ms": e0.elapsed_time(e1) / reps})
        plan.close()
    probe.close()
    if not timings:
        raise RuntimeError("no launch shape accepted for this scan")
    best = min(timings, key=lambda r: r["ms"])
    result = {"tile_cols": best["tile_cols"], "bin_groups": best["bin_groups"],
              "ms": best["ms"], "candidates": timings}
    if use_cache:
        store_cache(key, result)
    return dict(result, cached=False, key=key)


def tuned_plan(geom, wires, edges, images, **kw):
    """A Plan with the autotuned launch shape.  A cached shape tuned on a
    scan of the same class may not fit this one's shared memory (more steps
    in the same bucket); the scan is then tuned on its own.  A scan that
    takes the interval kernel (whose tile is fixed) is planned as it is."""
    plan_kw = {k: kw[k] for k in ("edge", "out_dtype", "geom_precision", "force_pixels")
               if k in kw}
    first = dr.Plan(geom, wires, edges, **plan_kw)
    if first.info()["kernel"] == "intervals":  # its tile shape is fixed: nothing to tune
        return first, {"tile_cols": first.info()["tile_cols"], "bin_groups": 0, "ms": None,
                       "candidates": [], "cached": False, "key": None}
    first.close()
    best = tune(geom, wires, edges, images, **kw)
    try:
        plan = dr.Plan(geom, wires, edges, tile_cols=best["tile_cols"],
                       bin_groups=best["bin_groups"], **plan_kw)
    except dr.DrError:
        if not best.get("cached"):
            raise
        kw = dict(kw, use_cache=False)
        best = tune(geom, wires, edges, images, **kw)
        plan = dr.Plan(geom, wires, edges, tile_cols=best["tile_cols"],
                       bin_groups=best["bin_groups"], **plan_kw)
    return plan, best


# (CTAs per SM, tile-width cap, threads per CTA)
BATCH_CANDIDATES = ((1, 0, 256), (1, 0, 512), (2, 0, 512), (2, 0, 256), (2, 64, 512),
                    (3, 0, 512), (3, 64, 512))


def tuned_batch(jobs, reps=2, stream=None):
    """The fastest batch build of these (plan, images, out) jobs: each
    candidate (CTAs per SM, tile-width cap) is built, replayed `reps` times
    and timed with CUDA events; the others are destroyed.  Returns
    (batch, timings)."""
    import torch

    stream = stream or torch.cuda.current_stream()
    best, timings, refused = None, [], []
    for per_sm, cap, nt in BATCH_CANDIDATES:
        try:
            b = dr.Batch(jobs, ctas_per_sm=per_sm, max_tile_cols=cap, threads=nt)
        except dr.DrError as e:
            refused.append(f"({per_sm}, {cap}, {nt}): {e}")
            continue
        b.launch(stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.launch(stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        timings.append({"ctas_per_sm": per_sm, "max_tile_cols": cap, "threads": nt, "ms": ms})
        if best is None or ms < best[0]:
            if best is not None:
                best[1].close()
            best = (ms, b, per_sm, cap, nt)
        else:
            b.close()
    if best is None:
        raise RuntimeError("no batch configuration accepted: " + "; ".join(refused))
    return best[1], {"ctas_per_sm": best[2], "max_tile_cols": best[3], "threads": best[4],
                     "candidates": timings}
