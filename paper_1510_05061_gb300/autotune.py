"""Autotuner for the batched and single-solve 3D steps: picks the tile shape
(TX x TY), the staging depth (synchronous loads, or the next plane copied
asynchronously one plane ahead: variants 4..7) and the z-chunk length
(planes marched per work item) by timing real steps with CUDA events on the
solve's stream.

The choice never changes results (every tile shape and chunk length gives
bit-identical states); it only changes speed.  Tuning advances the batch by
the steps it times.  Choices are cached per (GPU, precision, mode, workload
signature) in a JSON file (``HYDRO_AUTOTUNE_CACHE`` or
~/.cache/hydro_gb300/autotune.json).
"""

from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, Optional

from . import inputs

# longest z-chunk of an instance's column in a batch (shorter columns are one item)
DEFAULT_ZCHUNKS = (16, 32, 64, 128, 256)


def cache_path() -> str:
    return os.environ.get("HYDRO_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hydro_gb300", "autotune.json"))


_LIB_TAG = None


def lib_tag() -> str:
    """Short content hash of the loaded libhydro.so: a rebuilt library (new
    kernels) does not reuse choices timed on the old one."""
    global _LIB_TAG
    if _LIB_TAG is None:
        import hashlib

        from . import hydro

        try:
            with open(hydro.LIB_PATH, "rb") as fh:
                _LIB_TAG = hashlib.sha1(fh.read()).hexdigest()[:12]
        except OSError:
            _LIB_TAG = "unknown"
    return _LIB_TAG


def signature(batch) -> str:
    import torch

    probs = batch.probs
    p3 = [p for p in probs if p.ndim == 3]
    cells = sum(p.ncell for p in p3)
    ns = sorted(p.n[0] for p in p3)
    prec = "fp32" if probs[0].precision == inputs.FP32 else "fp64"
    hse = int(any(p.hse_subtract for p in p3))
    mag = f"{cells:.2g}" if cells else "0"
    span = f"{ns[0]}-{ns[-1]}" if ns else "none"
    return f"{torch.cuda.get_device_name()}|batch-v2|lib={lib_tag()}|{prec}|hse{hse}|n3d={len(p3)}|cells={mag}|n={span}"


def _load_cache() -> Dict[str, dict]:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(c: Dict[str, dict]):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_steps(batch, steps: int) -> float:
    """Milliseconds per step of the batch on its stream (CUDA events)."""
    import torch

    s = batch.stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    batch.step(steps)
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / steps


def tune_batch(batch, steps: int = 4, zchunks: Iterable[int] = DEFAULT_ZCHUNKS,
               variants: Optional[Iterable[int]] = None, use_cache: bool = True) -> dict:
    """Configure `batch` with the fastest (tile variant, z-chunk) and return
    the choice with the timing table."""
    from . import hydro

    key = signature(batch)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        ch = cache[key]
        batch.configure(ch["variant"], ch["zchunk"])
        return dict(ch, cached=True)
    shapes = hydro.batch_variants()
    variants = list(range(len(shapes))) if variants is None else list(variants)
    table = []
    best = None
    for v in variants:
        for z in zchunks:
            try:
                batch.configure(v, z)
            except hydro.HydroError:             # shape not available in this precision
                break
            batch.step(2)                        # first launch of this kernel, warm caches
            ms = time_steps(batch, steps)
            table.append({"variant": v, "tile": list(shapes[v]), "async_staging": v >= 4, "zchunk": z,
                          "ms_per_step": ms})
            if best is None or ms < best["ms_per_step"]:
                best = table[-1]
    batch.configure(best["variant"], best["zchunk"])
    choice = {"variant": best["variant"], "tile": best["tile"], "async_staging": best["async_staging"],
              "zchunk": best["zchunk"], "ms_per_step": best["ms_per_step"], "table": table}
    if use_cache:
        cache[key] = choice
        _store_cache(cache)
    return dict(choice, cached=False)


def sim_signature(sim) -> str:
    import torch

    p = sim.prob
    prec = "fp32" if p.precision == inputs.FP32 else "fp64"
    scheme = {inputs.SSPRK2: "rk2", inputs.CTU: "ctu"}.get(getattr(p, "scheme", 0), "hancock")
    if getattr(p, "recon", 0) == inputs.PPM:
        scheme += "-ppm"
    return (f"{torch.cuda.get_device_name()}|single-v2|lib={lib_tag()}|{prec}|hse{p.hse_subtract}|{scheme}"
            f"|n={p.n[0]}x{p.n[1]}x{p.n[2]}")


def time_sim_steps(sim, steps: int) -> float:
    import torch

    s = sim.stream
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    sim.run_steps(steps)
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / steps


def tune_simulation(sim, steps: int = 3, zchunks: Iterable[int] = (16, 32, 64, 128, -1, -64, -128),
                    variants: Optional[Iterable[int]] = None, use_cache: bool = True) -> dict:
    """Configure a single 3D solve with its fastest (tile shape, z-chunk);
    a negative z-chunk is the balanced grid (-1, hydro.ZCHUNK_BALANCED: over
    whole columns; -Z: over Z-plane chunks).  Tuning advances the solve by the
    steps it times."""
    from . import hydro

    if sim.prob.ndim != 3 or getattr(sim.prob, "scheme", 0) == inputs.CTU:
        # the 2D step and the corner transport upwind step have one launch shape
        return {"variant": 0, "tile": [32, 8], "zchunk": 1, "cached": False, "table": []}
    key = sim_signature(sim)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        ch = cache[key]
        sim.configure(ch["variant"], ch["zchunk"])
        return dict(ch, cached=True)
    shapes = dict(hydro.sim_variants())
    variants = sorted(shapes) if variants is None else list(variants)
    table, best = [], None
    for v in variants:
        for z in zchunks:
            if z > sim.prob.n[2]:
                continue
            try:
                sim.configure(v, z)
            except hydro.HydroError:
                break
            sim.run_steps(2)
            ms = time_sim_steps(sim, steps)
            table.append({"variant": v, "tile": list(shapes[v]), "async_staging": 4 <= v < 8,
                          "paired_cells": v in hydro.PAIR_VARIANTS, "zchunk": z, "ms_per_step": ms})
            if best is None or ms < best["ms_per_step"]:
                best = table[-1]
    sim.configure(best["variant"], best["zchunk"])
    choice = {"variant": best["variant"], "tile": best["tile"], "async_staging": best["async_staging"],
              "zchunk": best["zchunk"], "ms_per_step": best["ms_per_step"], "table": table}
    if use_cache:
        cache[key] = choice
        _store_cache(cache)
    return dict(choice, cached=False)
