"""Autotuner for the execution of a bootstrapping batch.

Candidates (all bit-identical in their results):
  * "grouped":    one launch per run of equal ring degree and variant, one
                  512-thread block per job;
  * "persistent": one launch for every job of degree 1024..4096, one
                  512-thread block per SM pulling jobs longest first.
Both are recorded in a CUDA graph and replayed.  The tuner times each
candidate on the batch itself and caches the winner in a JSON file keyed by
the GPU name and the batch composition (ring degree, rows per job, share).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import api

CANDIDATES = {"grouped": api.BATCH_GRAPH,
              "persistent": api.BATCH_GRAPH | api.BATCH_PERSISTENT}


def cache_path() -> str:
    return os.environ.get("BM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bootmmpm", "autotune.json"))


def signature(keys, jobs: np.ndarray, gpu_name: str) -> str:
    ns = np.array([keys[int(k)].kp.N for k in jobs["key"]])
    comp = {}
    for N, m in zip(ns, jobs["m"]):
        comp[f"{int(N)}x{int(m)}"] = comp.get(f"{int(N)}x{int(m)}", 0) + 1
    total = len(jobs)
    shares = ",".join(f"{k}:{round(v / total, 2)}" for k, v in sorted(comp.items()))
    size = 1 << int(np.log2(max(total, 1)))
    return f"{gpu_name}|{size}|{shares}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        with open(p + ".tmp", "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(p + ".tmp", p)
    except OSError:
        pass


def tune(keys, jobs, d_in, d_lut, d_out, ws, stream, reps: int = 1, use_cache: bool = True):
    """Returns (best candidate name, {name: ms}) for this batch."""
    import torch
    gpu = torch.cuda.get_device_name(stream.device)
    sig = signature(keys, jobs, gpu)
    cache = _load() if use_cache else {}
    if sig in cache:
        return cache[sig]["best"], cache[sig]["ms"]
    times = {}
    for name, flags in CANDIDATES.items():
        b = api.Batch([k.ek for k in keys], jobs, d_in, d_lut, d_out, ws, flags)
        b.run(stream)                      # records the graph
        stream.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        times[name] = best
        b.free()
    winner = min(times, key=times.get)
    cache[sig] = {"best": winner, "ms": times}
    if use_cache:
        _store(cache)
    return winner, times
