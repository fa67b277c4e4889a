"""Autotuner of the kernels' launch shapes (threads per block and resident
blocks per SM of the product kernel, selected per plan with
fofse_plan_set_variant).

It times every shape of every plan on the caller's own batch with CUDA events
and keeps the fastest; choices are cached in a JSON file keyed by the GPU
name, the plan's parameters and the batch size (rounded to a power of two),
so a workload is timed once per machine.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api
from . import binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
_lock = threading.Lock()


def _key(plan, n_blocks, device):
    name = torch.cuda.get_device_name(device)
    bucket = 1 << max(0, int(n_blocks) - 1).bit_length()
    return (f"{name}|T{plan.fft_size}|b{plan.block}|br{plan.border}|I{plan.iters}|"
            f"{plan.precision}|s{plan.support}|c{getattr(plan, 'compensation', 0)}|basis{getattr(plan, 'basis', 0)}|n{bucket}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(plans, blocks, frame, avail, *, reps: int = 3, use_cache: bool = True,
             cache_path: str = CACHE, stream=None) -> dict:
    """Select the fastest launch shape of every plan for this batch.  Returns
    {"choices": [variant per plan], "timings_ms": [...], "cached": [bool]}."""
    plans = list(plans)
    n = int(blocks.shape[0])
    dev = frame.device
    stream = stream or torch.cuda.current_stream(dev)
    with _lock:
        cache = _load(cache_path) if use_cache else {}
    choices, timings, cached = [], [], []
    ob, tr, w0, st = api.alloc_outputs(plans, n, dev)
    ws = api.workspace(plans, n, dev)
    handles = [p.handle for p in plans]

    def run():
        B.fofse_extrapolate_batch(handles, blocks, frame, avail, out_blocks=ob, trace=tr, w0=w0,
                                  status=st, workspace=ws, stream=stream)

    for p in plans:
        count = B.fofse_plan_variant_count(p.handle)
        key = _key(p, n, dev)
        if use_cache and key in cache and 0 <= cache[key]["variant"] < count:
            B.fofse_plan_set_variant(p.handle, cache[key]["variant"])
            choices.append(cache[key]["variant"])
            timings.append(cache[key]["ms"])
            cached.append(True)
            continue
        ms = []
        for v in range(count):
            B.fofse_plan_set_variant(p.handle, v)
            run()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1) / reps)
        best = min(range(count), key=lambda v: ms[v])
        B.fofse_plan_set_variant(p.handle, best)
        choices.append(best)
        timings.append(ms)
        cached.append(False)
        cache[key] = {"variant": best, "ms": ms}
    B.fofse_check(stream)
    if use_cache:
        with _lock:
            merged = _load(cache_path)
            merged.update(cache)
            _save(cache_path, merged)
    return {"choices": choices, "timings_ms": timings, "cached": cached}


def _volume_key(plan, n_blocks, device):
    name = torch.cuda.get_device_name(device)
    bucket = 1 << max(0, int(n_blocks) - 1).bit_length()
    return (f"{name}|volume|T{plan.fft_size}x{plan.fft_time}|b{plan.block}|br{plan.border}|"
            f"d{plan.depth}|I{plan.iters}|{plan.precision}|n{bucket}")


def autotune_volume(plan, blocks, video, avail, *, reps: int = 3, use_cache: bool = True,
                    cache_path: str = CACHE, stream=None) -> dict:
    """Select the fastest launch shape of a volume plan (FP32 kernel) for this
    batch.  Returns {"choice": variant, "timings_ms": [...], "cached": bool}."""
    n = int(blocks.shape[0])
    dev = video.device
    stream = stream or torch.cuda.current_stream(dev)
    count = B.fofse_volume_plan_variant_count(plan.handle)
    key = _volume_key(plan, n, dev)
    with _lock:
        cache = _load(cache_path) if use_cache else {}
    if use_cache and key in cache and 0 <= cache[key]["variant"] < count:
        B.fofse_volume_plan_set_variant(plan.handle, cache[key]["variant"])
        return {"choice": cache[key]["variant"], "timings_ms": cache[key]["ms"], "cached": True}
    out = torch.empty((n, plan.block, plan.block), dtype=torch.float32, device=dev)
    ws = api.volume_workspace(plan, n, dev)
    ms = []
    for v in range(count):
        B.fofse_volume_plan_set_variant(plan.handle, v)

        def run():
            B.fofse_extrapolate_volume_batch(plan.handle, blocks, video, avail, out_blocks=out,
                                             workspace=ws, stream=stream)
        run()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(max(reps, 5)):  # the median of single launches
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        ms.append(sorted(ts)[len(ts) // 2])
    B.fofse_check(stream)
    # the default shape unless another is clearly faster (the shapes of a grid
    # are often within a few per cent of each other, inside the noise of a few
    # launches)
    best = min(range(count), key=lambda v: ms[v])
    if ms[best] > 0.97 * ms[0]:
        best = 0
    B.fofse_volume_plan_set_variant(plan.handle, best)
    if use_cache:
        with _lock:
            merged = _load(cache_path)
            merged[key] = {"variant": best, "ms": ms}
            _save(cache_path, merged)
    return {"choice": best, "timings_ms": ms, "cached": False}
