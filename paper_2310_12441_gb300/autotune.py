"""Autotuner of bootstrapping batches on one GPU.

Two choices, both bit-identical in their results (every candidate computes
Algorithm 1 exactly; tests/test_gpu_shapes.py checks each against the
oracle):

  * the kernel shape of each ring degree in the batch (bm_kernel_shape_info:
    NTT radix 16 or 8, 256 / 512 / 1024 threads per block, one or two blocks
    per SM), timed on a sample of the batch's jobs of that degree;
  * the launch mode: "grouped" (one launch per run of equal degree and
    arithmetic variant, one after the other) or "persistent" (one persistent
    kernel per such class, the classes running concurrently), timed on the
    whole batch with the chosen shapes.

Every candidate is recorded in a CUDA graph once and timed over `reps`
replays (the minimum counts).  The winner is cached in a JSON file keyed by
the GPU's name, the library's build (hash of libbootmmpm.so) and the batch
composition (ring degree and rows per job, their shares, batch size bucket),
and applied with bm_set_kernel_shape.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import api

MODES = {"grouped": api.BATCH_GRAPH,
         "persistent": api.BATCH_GRAPH | api.BATCH_PERSISTENT}
# kept for callers that iterate over the launch modes
CANDIDATES = MODES


def cache_path() -> str:
    return os.environ.get("BM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bootmmpm", "autotune.json"))


def library_hash() -> str:
    h = hashlib.sha256()
    with open(api.library_path(), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def signature(keys, jobs: np.ndarray, gpu_name: str) -> str:
    ns = np.array([keys[int(k)].kp.N for k in jobs["key"]])
    comp = {}
    for N, m in zip(ns, jobs["m"]):
        comp[f"{int(N)}x{int(m)}"] = comp.get(f"{int(N)}x{int(m)}", 0) + 1
    total = len(jobs)
    shares = ",".join(f"{k}:{round(v / total, 2)}" for k, v in sorted(comp.items()))
    size = 1 << int(np.log2(max(total, 1)))
    return f"{gpu_name}|{library_hash()}|{size}|{shares}"


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


def _time_batch(keys, jobs, d_in, d_lut, d_out, ws, flags, stream, reps) -> float:
    import torch
    b = api.Batch(keys, jobs, d_in, d_lut, d_out, ws, flags)
    try:
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
        return best
    finally:
        b.free()


def apply(result: dict) -> None:
    for N, d in result["shapes"].items():
        api.set_kernel_shape(int(N), int(d["choice"]))


def tune(keysets, jobs, d_in, d_lut, d_out, ws, stream, reps: int = 3, use_cache: bool = True,
         sample: int = 608) -> dict:
    """Tunes the batch (keysets: objects with .ek and .kp; jobs: api.JOB_DTYPE).
    Returns {"shapes": {N: {"choice", "ms": {shape: ms}, "runner_up"}},
    "mode": name, "mode_ms": {name: ms}} and applies the shapes."""
    import torch
    keys = [k.ek for k in keysets]
    gpu = torch.cuda.get_device_name(stream.device)
    sig = signature(keysets, jobs, gpu)
    cache = _load() if use_cache else {}
    if sig in cache:
        apply(cache[sig])
        return cache[sig]
    Ns = np.array([keysets[int(k)].kp.N for k in jobs["key"]])
    result = {"shapes": {}, "mode": None, "mode_ms": {}}
    for N in sorted(set(int(x) for x in Ns)):
        sel = np.nonzero(Ns == N)[0]
        if len(sel) > sample:                   # an even sample of this degree's jobs
            sel = sel[np.linspace(0, len(sel) - 1, sample).astype(int)]
        sub = jobs[sel]
        times = {}
        if not api.kernel_shapes(N):            # ring degrees above 8192: no shape choice
            continue
        for sh in api.kernel_shapes(N):
            api.set_kernel_shape(N, sh)
            times[sh] = _time_batch(keys, sub, d_in, d_lut, d_out, ws, api.BATCH_GRAPH, stream, reps)
        order = sorted(times, key=times.get)
        api.set_kernel_shape(N, order[0])
        result["shapes"][N] = {"choice": order[0], "ms": times, "jobs_timed": int(len(sel)),
                               "runner_up": order[1] if len(order) > 1 else None,
                               "desc": {sh: api.kernel_shapes(N)[sh] for sh in times}}
    for name, flags in MODES.items():
        result["mode_ms"][name] = _time_batch(keys, jobs, d_in, d_lut, d_out, ws, flags, stream, reps)
    result["mode"] = min(result["mode_ms"], key=result["mode_ms"].get)
    if use_cache:
        cache = _load()
        cache[sig] = json.loads(json.dumps(result))     # JSON keys: ring degrees and shapes as strings
        _store(cache)
    return result
