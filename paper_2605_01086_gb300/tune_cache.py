"""Persistent cache of autotuned plan options.

``fptc_plan_autotune`` times the candidate kernels, tile sizes and CTA shapes on
the caller's own batch.  ``tuned_plan`` keeps the winner in a small JSON file,
keyed by the GPU's name, the transform precision, the set of domain shapes
(N, E, L_max) and power-of-two size classes of the batch (samples and streams),
so that a later plan for a similar batch on the same kind of GPU starts with
those options instead of tuning again.  The decoder itself is stateless; this file is the only state kept
between runs, and a missing or unreadable file just means tuning again.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

from . import _lib

_NAMES = {
    "idct": {v: k for k, v in _lib.IDCT.items()},
    "schedule": {v: k for k, v in _lib.SCHEDULE.items()},
    "kernel": {v: k for k, v in _lib.KERNEL.items()},
}


def cache_key(gpu_name: str, domains, n_samples: int, n_segments: int, idct: str = "fp32") -> str:
    """Key of a batch: GPU name, transform precision, sorted distinct (N, E, L_max)
    of its domains, and floor(log2) of its sample and stream counts."""
    shapes = sorted({(int(d.N), int(d.E), int(d.lmax)) for d in domains})
    s_class = int(math.log2(n_samples)) if n_samples > 0 else -1
    n_class = int(math.log2(n_segments)) if n_segments > 0 else -1
    return json.dumps([gpu_name, idct, shapes, s_class, n_class])


def plan_kwargs(options: dict) -> dict:
    """Plan constructor arguments from the integer options fptc_plan_autotune returns."""
    kw = {}
    for k in ("idct", "schedule", "kernel"):
        if k in options:
            kw[k] = _NAMES[k][int(options[k])]
    for k in ("tile_samples", "threads", "ctas_per_sm"):
        if k in options:
            kw[k] = int(options[k])
    return kw


class TuneCache:
    """The JSON file: {key: {"options": {...}, "ms": float}}."""

    def __init__(self, path: str):
        self.path = path
        self.entries = {}
        try:
            with open(path) as f:
                data = json.load(f)
            if isinstance(data, dict):
                self.entries = {k: v for k, v in data.items()
                                if isinstance(v, dict) and isinstance(v.get("options"), dict)}
        except (OSError, ValueError):
            self.entries = {}

    def get(self, key: str):
        e = self.entries.get(key)
        return None if e is None else dict(e["options"])

    def put(self, key: str, options: dict, ms: float):
        self.entries[key] = {"options": {k: int(v) for k, v in options.items()}, "ms": float(ms)}
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tune_cache.", dir=d)
        with os.fdopen(fd, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)  # a reader sees the old file or the new one, never a torn one


def tuned_plan(domains, segments, words, symlen, cache_path: str, device=None, idct: str = "fp32", trials: int = 3,
               plan_cls=None, gpu_name=None):
    """A decode Plan with tuned options: from the cache when the batch's key is
    there, else tuned on (words, symlen) and stored.  Returns (plan, options,
    hit).  plan_cls and gpu_name default to Plan and the device's name."""
    if plan_cls is None:
        from .decoder import Plan as plan_cls
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name(device)
    n_samples = int(sum(int(s["n_samples"]) for s in segments))
    key = cache_key(gpu_name, domains, n_samples, len(segments), idct)
    cache = TuneCache(cache_path)
    hit = cache.get(key)
    if hit is not None:
        return plan_cls(domains, segments, device=device, **plan_kwargs(hit)), hit, True
    plan = plan_cls(domains, segments, device=device, idct=idct)
    out = plan.empty_out()
    best, ms = plan.autotune(words, symlen, out, trials=trials)
    cache.put(key, best, ms)
    return plan, best, False
