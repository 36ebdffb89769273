"""Benchmark: BootMMPM bootstraps/s on one GB300 (batched vs plain, bit-exact),
with p50/p99 served latency.

One step = one batch of the workload (default: 4096 ciphertexts, n = 630,
N = 1024, m = 4, t = 2^10) through the whole hot path: test vector and ACC
initialisation, n CMux steps, sample extraction, key switching.  Keys are
generated on the device from a seed.  Every warm-up and timed step bootstraps
its own freshly encrypted batch (distinct ciphertexts and tables), all
resident in HBM before the timed region; every output of every step is
decrypted afterwards and counted in `decrypt_failures`.  L2 is flushed
between timed steps (the keys, 236 MiB BSK and 518 MiB KSK, exceed L2 too).

Also reported in the same JSON line: the plain form (one ciphertext per
launch), the end-to-end rate through the host-buffer C-ABI call, the
blind-rotation kernel's integer roofline, SM clocks during the timed region,
the key switch's gather bandwidth, the large-plaintext (n = 750, N = 2048,
m = 8) and single-polynomial (m = 1, N = 4096) workloads with their roofline
fractions, the uneven mix in grouped and persistent launches, served p50/p99
latency at three loads, and the CPU oracle's rate on a bounded sample
(`--impl reference` prints the oracle arm alone).

Multi-GPU: independent replicas (weak scaling), one process per GPU under
torchrun; each rank bootstraps its own batches; value = total / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_12441_gb300 import params as P  # noqa: E402
from paper_2310_12441_gb300 import synth  # noqa: E402

METRIC = "bootstraps/s on 1 GB300 (batched vs plain, bit-exact); p50/p99 served latency"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the
# blind-rotation kernel per job, from one ncu capture of a 152-job launch of
# the workload (command: bench.py --workload <name> --count 152 under
# `ncu --set full -k regex:k_blind_rotate`), valid while the kernel sources
# hash to the captured version.
KERNEL_SOURCES = ["blind_rotate.cuh", "ntt_reg.cuh", "modarith.cuh", "common.cuh", "br_launch.cuh"]
CAPTURED_TRAFFIC = {
    P.BATCH_N1024.name: {"hash": "2e5795488aa486bf", "bytes_per_job": (254.637056e6 + 6.749184e6) / 152},
}


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2310_12441_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def modmuls_per_bootstrap(kp, m):
    """Algorithmic 64-bit modular multiplications of one bootstrap: per CMux
    step and row, 4 l_B forward and 2 inverse negacyclic NTTs of (N/2) log2 N
    butterflies, and 8 l_B N multiply-accumulates against the key."""
    import math
    N, lB = kp.N, kp.l_B
    return kp.n * m * ((4 * lB + 2) * (N // 2) * int(math.log2(N)) + 8 * lB * N)


class ClockSampler:
    """Samples nvidia-smi during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7
                          for i in range(4) if r[3 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


def aggregate(local_ms: float, count_per_rank: int, steps: int, world: int, dist=None, device=None):
    """Whole-job rate over replicas: every rank bootstraps its own batch
    (weak scaling); the job takes as long as the slowest rank, so the total
    time is the maximum over ranks and the rate counts all ranks' work."""
    total_ms = float(local_ms)
    if world > 1 and dist is not None:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, count_per_rank * world * steps / (total_ms * 1e-3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------

def oracle_rate(w, cores_hint=None, steps_sample=8, seed=0):
    """The oracle on a bounded sample of the workload: `cores` ciphertexts,
    one per core, whose masks vanish after the first `steps_sample` entries
    (so the oracle runs only those CMux steps), each followed by its full key
    switch.  Returns the measured wall time of the sample and the rate it
    projects for full bootstraps (CMux steps all cost the same, so the
    rotation time scales by n / steps_sample; the key switch is timed alone)."""
    import oracle
    kp, m, t = w.keys, w.shape.m, w.shape.t
    cores = cores_hint or os.cpu_count() or 1
    S = cores
    rnd = oracle.seeded_key_randomness(kp, 1000 + w.seed_base, bsk_keys=steps_sample)
    bsk = oracle.keygen_bsk(kp, rnd)
    ksk = oracle.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = synth.messages(t, S, 3000 + w.seed_base + seed)
    ct = oracle.encrypt_seeded(kp.n, qp, t, rnd["s"], msg, kp.sigma, 4000 + w.seed_base + seed)
    ct[:, steps_sample:kp.n] = 0
    luts, _ = synth.luts(t, S, 2000 + w.seed_base + seed)
    t0 = time.perf_counter()
    oracle.bootstrap(kp, m, t, bsk, ksk, ct, luts)
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    lwe = np.zeros((S, kp.N + 1), np.uint64)
    for i in range(S):
        oracle.key_switch(kp, lwe[i], ksk)
    ks = (time.perf_counter() - t1) / S          # serial, one core
    per_ct_rot = max(dt - ks, 1e-9)              # wall, S in parallel
    per_boot_wall = per_ct_rot * kp.n / steps_sample + ks
    rate = S / per_boot_wall
    sample = (f"{S} ciphertexts (one per core) x first {steps_sample} of {kp.n} CMux steps "
              f"+ full key switch: {dt:.2f} s wall measured; full bootstraps/s projected "
              f"by scaling the rotation time to n steps")
    return rate, cores, sample, dt


def run_reference(args, w):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    for s in range(args.warmup):                  # untimed: loads the library, warms caches
        oracle_rate(w, steps_sample=1, seed=100 + s)
    vals, walls = [], []
    for s in range(args.steps):
        r, cores, sample, dt = oracle_rate(w, steps_sample=args.cpu_steps, seed=s)
        vals.append(r)
        walls.append(dt)
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "bootstraps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(walls)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config_of(w, args),
            "step": "one bounded sample of the workload (see cpu_baseline.sample); ms_per_step "
                    "is its measured wall time",
            "projected_bootstraps_per_s": v,
            "projected_ms_per_batch": 1e3 * (args.count or w.count) / v,
            "cpu_baseline": {"value": v, "unit": "bootstraps/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "bootstraps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w, args, count=None):
    kp = w.keys
    return {"workload": w.name, "count": count or args.count or w.count, "n": kp.n, "N": kp.N,
            "m": w.shape.m, "t": w.shape.t, "Q": kp.Q, "B": kp.B, "l_B": kp.l_B,
            "B_ks": kp.Bks, "l_ks": kp.l_ks, "keys": "drawn and built on the device from a seed",
            "inputs": "a distinct encrypted batch per step, resident before timing",
            "l2": "flushed between timed steps", "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def make_inputs(api, sk, w, count, seed, dev):
    """One batch: messages, tables and seeded encryptions, copied to `dev`."""
    import torch
    kp, m, t = w.keys, w.shape.m, w.shape.t
    qp = 2 * kp.N * m
    luts, ident = synth.luts(t, count, 2000 + seed, mix=w.lut_mix)
    msg = synth.messages(t, count, 3000 + seed, half=ident)
    ct = api.bm_encrypt_seeded(sk, qp, t, msg, 4000 + seed)
    return {"ct": ct, "luts": luts, "d_in": api.to_device_u64(ct.ravel(), dev),
            "d_lut": api.to_device_u32(luts.ravel(), dev),
            "d_out": torch.zeros(count * (kp.n + 1), dtype=torch.int64, device=dev)}


def count_failures(api, sk, w, batches):
    """Outputs that do not decrypt (at Q) to f(Dec(input))."""
    kp, m, t = w.keys, w.shape.m, w.shape.t
    qp, W = 2 * kp.N * m, kp.n + 1
    bad = total = 0
    for b in batches:
        cnt = b["ct"].shape[0]
        out = api.from_device_u64(b["d_out"]).reshape(cnt, W)
        dec_in = api.bm_decrypt(sk, qp, t, b["ct"])
        dec_out = api.bm_decrypt(sk, kp.Q, t, out)
        bad += int((dec_out != b["luts"][np.arange(cnt), dec_in]).sum())
        total += cnt
    return bad, total


def kernel_roofline(api, ek, w, jobs, batch, ws, stream, flush, dev, peak, reps=3):
    """Blind rotation alone (bm_blind_rotate, same jobs and launch shape)
    timed with CUDA events on its stream: algorithmic modmuls / time against
    the measured modmul peak."""
    import torch
    kp, m = w.keys, w.shape.m
    count = len(jobs)
    d_acc = torch.zeros(count * 2 * m * kp.N, dtype=torch.int64, device=dev)
    jobs_acc = jobs.copy()
    jobs_acc["out_off"] = np.arange(count) * 2 * m * kp.N
    ts = []
    for _ in range(reps):
        flush.fill_(1)
        a, b = _events(torch)
        a.record(stream)
        api.bm_blind_rotate([ek], jobs_acc, 1 << 30, batch["d_in"], batch["d_lut"], d_acc, ws, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    del d_acc
    mm = modmuls_per_bootstrap(kp, m) * count
    rot_s = float(np.mean(ts)) * 1e-3
    traffic = None
    cap = CAPTURED_TRAFFIC.get(w.name)
    if cap and kernel_hash() == cap["hash"]:
        traffic = cap["bytes_per_job"] * count
    shape = api.get_kernel_shape(kp.N)
    radix, threads, blocks = api.kernel_shapes(kp.N)[shape]
    return {"bound": "alu", "achieved": mm / rot_s / 1e9, "peak": peak / 1e9, "unit": "Gmodmul/s",
            "frac": (mm / rot_s) / peak, "traffic": traffic, "kernel": "k_blind_rotate",
            "shape": {"id": shape, "ntt_radix": radix, "threads": threads, "blocks_per_sm": blocks},
            "kernel_ms": rot_s * 1e3, "modmuls_per_launch": mm,
            "peak_kind": "measured: the blind rotation's own modular product in a throughput loop"}


def run_workload(api, w, dev, stream, flush, peak, count=None, steps=2, warmup=1, seed_shift=0):
    """Rate, roofline and failures of one more workload (its own keys)."""
    import torch
    kp, m, t = w.keys, w.shape.m, w.shape.t
    count = count or w.count
    t0 = time.perf_counter()
    sk, ek = api.bm_keygen_seeded(kp, 1000 + w.seed_base, dev.index)
    torch.cuda.synchronize(dev)
    keygen_s = time.perf_counter() - t0
    W = kp.n + 1
    jobs = api.make_jobs(0, m, t, np.arange(count) * W, np.arange(count) * t, np.arange(count) * W)
    ws = api.workspace(api.bm_workspace_bytes([ek], jobs), dev)
    batches = [make_inputs(api, sk, w, count, w.seed_base + 700 + seed_shift + i, dev)
               for i in range(warmup + steps)]
    for b in batches[:warmup]:
        api.bm_bootstrap_batch([ek], jobs, b["d_in"], b["d_lut"], b["d_out"], ws, stream)
    torch.cuda.synchronize(dev)
    ms = []
    for b in batches[warmup:]:
        flush.fill_(4)
        e0, e1 = _events(torch)
        e0.record(stream)
        api.bm_bootstrap_batch([ek], jobs, b["d_in"], b["d_lut"], b["d_out"], ws, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    assert api.bm_workspace_status(ws, stream) == 0
    bad, total = count_failures(api, sk, w, batches)
    roof = kernel_roofline(api, ek, w, jobs, batches[0], ws, stream, flush, dev, peak, reps=1)
    value = count / (float(np.mean(ms)) * 1e-3)
    del batches, ws
    ek.free()
    torch.cuda.empty_cache()
    return {"workload": w.name, "value": value, "unit": "bootstraps/s", "ms_per_step": float(np.mean(ms)),
            "steps": steps, "count": count, "keygen_s": keygen_s, "key_bytes": None,
            "decrypt_failures": bad, "bootstraps_checked": total, "roofline": roof}


def key_switch_rate(api, ek, kp, count, dev, stream, flush, hbm_gbs):
    """bm_key_switch on `count` random LWE_{N,Q} samples: the selected KSK rows
    (digits nonzero: 15/16 of N l_ks per sample, n + 1 words each) per second,
    against the measured HBM copy bandwidth."""
    import torch
    rng = np.random.default_rng(5)
    lwe = rng.integers(0, kp.Q, (count, kp.N + 1), dtype=np.uint64)
    d_in = api.to_device_u64(lwe, dev)
    d_out = torch.zeros(count * (kp.n + 1), dtype=torch.int64, device=dev)
    api.bm_key_switch(ek, d_in, count, d_out, stream)
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(3):
        flush.fill_(5)
        a, b = _events(torch)
        a.record(stream)
        api.bm_key_switch(ek, d_in, count, d_out, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    rows = kp.N * kp.l_ks * (kp.Bks - 1) / kp.Bks * count
    gbytes = rows * (kp.n + 1) * 8 / 1e9
    ksk_bytes = kp.N * kp.l_ks * (kp.Bks - 1) * (kp.n + 1) * 8
    one = []
    for _ in range(3):
        a, b = _events(torch)
        a.record(stream)
        api.bm_key_switch(ek, d_in, 1, d_out, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        one.append(a.elapsed_time(b))
    return {"kernel": "key switch (bm_key_switch)", "count": count, "ms": ms,
            "gathered_gbytes": gbytes, "gathered_GBps": gbytes / (ms * 1e-3),
            "ksk_bytes": ksk_bytes, "hbm_peak_GBps": hbm_gbs,
            "frac_gathered_of_hbm": gbytes / (ms * 1e-3) / hbm_gbs if hbm_gbs else None,
            "single_ms": float(np.median(one))}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def run_gpu(args, w):
    import torch
    import torch.distributed as dist

    from paper_2310_12441_gb300 import api

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kp, m, t = w.keys, w.shape.m, w.shape.t
    count = args.count or w.count
    api.load(build_if_needed=(rank == 0))

    t0 = time.perf_counter()
    sk, ek = api.bm_keygen_seeded(kp, 1000 + w.seed_base, local)
    torch.cuda.synchronize(dev)
    keygen_s = time.perf_counter() - t0
    W = kp.n + 1
    jobs = api.make_jobs(0, m, t, np.arange(count) * W, np.arange(count) * t, np.arange(count) * W)
    seed = w.seed_base + 100 * rank
    batches = [make_inputs(api, sk, w, count, seed + 1000 * i, dev) for i in range(args.warmup + args.steps)]
    ws = api.workspace(api.bm_workspace_bytes([ek], jobs), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(b):
        api.bm_bootstrap_batch([ek], jobs, b["d_in"], b["d_lut"], b["d_out"], ws, stream)

    for b in batches[:args.warmup]:
        step(b)
    torch.cuda.synchronize(dev)
    assert api.bm_workspace_status(ws, stream) == 0

    evs = [_events(torch) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            step(batches[args.warmup + i])
            evs[i][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms, value = aggregate(float(sum(ms)), count, args.steps, world, dist if world > 1 else None, dev)
    assert api.bm_workspace_status(ws, stream) == 0
    failures, checked = count_failures(api, sk, w, batches)
    timed_failures, timed_checked = count_failures(api, sk, w, batches[args.warmup:])

    result = {"metric": METRIC, "value": value, "unit": "bootstraps/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
              "data": "synthetic", "config": config_of(w, args),
              "decrypt_failures": timed_failures, "bootstraps_checked": timed_checked,
              "decrypt_failures_incl_warmup": failures, "bootstraps_checked_incl_warmup": checked,
              "gpu_launches": 2 * args.steps, "keygen_s": keygen_s}
    if rank == 0:
        result["clocks"] = clk.summary()
        peaks = measured_peaks()
        peak = api.bm_modmul_peak(local, 1 << 14)
        result["roofline"] = kernel_roofline(api, ek, w, jobs, batches[0], ws, stream, flush, dev, peak)
        # plain form: one ciphertext per launch
        if args.plain > 0:
            b0 = batches[0]
            P_ = min(args.plain, count)
            j1 = [jobs[i:i + 1] for i in range(P_)]
            for i in range(2):
                api.bm_bootstrap_batch([ek], j1[i], b0["d_in"], b0["d_lut"], b0["d_out"], ws, stream)
            torch.cuda.synchronize(dev)
            a, b = _events(torch)
            a.record(stream)
            for i in range(P_):
                api.bm_bootstrap_batch([ek], j1[i], b0["d_in"], b0["d_lut"], b0["d_out"], ws, stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            pv = P_ / (a.elapsed_time(b) * 1e-3)
            P1 = min(8, P_)
            d_out1 = torch.zeros_like(b0["d_out"])
            one = [api.Batch([ek], j1[i], b0["d_in"], b0["d_lut"], d_out1, ws, api.BATCH_ONE_BLOCK)
                   for i in range(P1)]
            one[0].run(stream)
            torch.cuda.synchronize(dev)
            a.record(stream)
            for bt in one:
                bt.run(stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            pv1 = P1 / (a.elapsed_time(b) * 1e-3)
            for bt in one:
                bt.free()
            result["plain"] = {"value": pv, "unit": "bootstraps/s", "ciphertexts": P_,
                               "batched_over_plain": value / pv,
                               "launch": "one job per launch, rows split over a thread-block cluster",
                               "one_block_per_job": {"value": pv1, "ciphertexts": P1}}
        # end to end through the host-buffer C-ABI call (pinned host memory)
        b0 = batches[0]
        h_in = torch.from_numpy(b0["ct"].ravel().view(np.int64)).pin_memory()
        h_lut = torch.from_numpy(b0["luts"].ravel().view(np.int32)).pin_memory()
        h_out = torch.zeros(count * W, dtype=torch.int64).pin_memory()
        ws2 = api.workspace(api.bm_workspace_bytes([ek], jobs) + api.bm_host_staging_bytes([ek], jobs) + 4096, dev)
        api.bm_bootstrap_batch_host([ek], jobs, h_in, h_lut, h_out, ws2, stream)
        e2e_ms = []
        for i in range(max(1, min(args.steps, 3))):
            flush.fill_(2)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            api.bm_bootstrap_batch_host([ek], jobs, h_in, h_lut, h_out, ws2, stream)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del ws2
        result["e2e"] = {"value": count / (np.mean(e2e_ms) * 1e-3), "unit": "bootstraps/s",
                         "h2d_bytes_per_step": int(h_in.numel() * 8 + h_lut.numel() * 4),
                         "d2h_bytes_per_step": int(h_out.numel() * 8)}
        result["key_switch"] = key_switch_rate(api, ek, kp, count, dev, stream, flush, peaks.get("hbm_gbs"))
        if not args.no_extras and w is P.BATCH_N1024:
            del batches
            torch.cuda.empty_cache()
            result.update(run_extras(args, api, dev, stream, flush, peak))
            # decryption failures over at least --fail-count bootstraps of this
            # run: every output above, then further (untimed) headline batches
            tot, bad = checked, failures
            for wr in result["workloads"]:
                tot += wr["bootstraps_checked"]
                bad += wr["decrypt_failures"]
            n_uneven = sum(result["uneven"]["counts"].values())
            for md in result["uneven"]["modes"].values():
                tot += n_uneven
                bad += md["decrypt_failures"]
            extra = 0
            while tot < args.fail_count:
                b = make_inputs(api, sk, w, count, seed + 1000 * (args.warmup + args.steps + extra), dev)
                step(b)
                torch.cuda.synchronize(dev)
                f, c = count_failures(api, sk, w, [b])
                tot += c
                bad += f
                extra += 1
                del b
            result["failures"] = {"bootstraps": tot, "decrypt_failures": bad,
                                  "of": "every output of this run (headline incl. warm-up, other workloads, "
                                        f"uneven mix) plus {extra} further headline batches"}
        if not args.no_cpu:
            r, cores, sample, _ = oracle_rate(w, steps_sample=args.cpu_steps)
            result["cpu_baseline"] = {"value": r, "unit": "bootstraps/s", "cores": cores,
                                      "kind": "oracle", "sample": sample}
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_extras(args, api, dev, stream, flush, peak):
    """The other workloads of the metric, inside the same JSON line: the
    large-plaintext and single-polynomial batches (rate and roofline), the
    uneven mix in grouped and persistent launches, and served latency."""
    import torch
    from paper_2310_12441_gb300 import autotune, serve
    from paper_2310_12441_gb300 import workload as wl
    from paper_2310_12441_gb300.params import JobShape
    out = {"workloads": []}
    stream = torch.cuda.Stream(dev)     # graph capture needs a stream other than the legacy default
    for w2 in (P.LARGE_N2048, P.SINGLEPOLY_N4096):
        out["workloads"].append(run_workload(api, w2, dev, stream, flush, peak))
    # uneven mix: 8192 jobs over six parameter sets, Zipf(1.2) counts
    ks1024 = wl.make_keyset(P.KEYS_N1024, 1002)
    ks2048 = wl.make_keyset(P.KEYS_N2048, 1003)
    ksets = [ks1024, ks2048]
    counts = synth.zipf_counts(8192, len(P.UNEVEN_SETS), 1.2, 5)
    groups = [(0 if kp is P.KEYS_N1024 else 1, shape, int(c))
              for (name, kp, shape), c in zip(P.UNEVEN_SETS, counts)]
    bu = wl.make_batch(ksets, groups, 4)
    d_in = api.to_device_u64(bu.ct_in, dev)
    d_lut = api.to_device_u32(bu.luts, dev)
    d_out = torch.zeros(bu.out_words, dtype=torch.int64, device=dev)
    keys = [k.ek for k in ksets]
    ws = api.workspace(api.bm_workspace_bytes(keys, bu.jobs), dev)
    tuned = autotune.tune(ksets, bu.jobs, d_in, d_lut, d_out, ws, stream, use_cache=False)
    modes = {}
    mm = sum(modmuls_per_bootstrap(ksets[int(j["key"])].kp, int(j["m"])) for j in bu.jobs)
    for name, fl in autotune.CANDIDATES.items():
        b = api.Batch(keys, bu.jobs, d_in, d_lut, d_out, ws, fl)
        b.run(stream)
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(2):
            flush.fill_(6)
            e0, e1 = _events(torch)
            e0.record(stream)
            b.run(stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        b.free()
        ms = float(np.min(ts))
        bad = wl.check_outputs(ksets, bu, api.from_device_u64(d_out))
        modes[name] = {"bootstraps_per_s": len(bu.jobs) / ms * 1e3, "ms": ms, "decrypt_failures": bad,
                       "frac_of_modmul_peak": mm / (ms * 1e-3) / peak}
    out["uneven"] = {"workload": "uneven 8192 jobs, sets S1..S6 (m 1..8, N 1024/2048), Zipf 1.2",
                     "counts": {n: int(c) for (n, _, _), c in zip(P.UNEVEN_SETS, counts)},
                     "autotune": tuned, "modes": modes}
    for N in (1024, 2048, 4096):
        api.set_kernel_shape(N, api.SHAPE_DEFAULT)
    del d_in, d_lut, d_out, ws, bu
    # served: single requests of the large-plaintext set at fractions of its batch capacity
    cap = out["workloads"][0]["value"]
    poolsz = 512
    bp = wl.make_batch([ks2048], [(0, JobShape(8, 8192), poolsz)], 9, lut_mix="mixed", interleave=False)
    Wn = P.KEYS_N2048.n + 1
    pool = [(0, 8, 8192, bp.ct_in[i * Wn:(i + 1) * Wn], bp.luts[i * 8192:(i + 1) * 8192])
            for i in range(poolsz)]
    served = []
    for frac in (0.25, 0.5, 0.9):
        srv = serve.Server([ks2048], max_batch=args.max_batch, streams=3)
        r = serve.run_open_loop(srv, pool, frac * cap, args.serve_seconds, 11)
        r.pop("requests")
        r["load"] = frac
        served.append(r)
    out["served"] = {"workload": "Poisson arrivals of single requests, n=750 N=2048 m=8 t=2^13, "
                                 "random and identity tables", "capacity_bootstraps_per_s": cap,
                     "memory_cap_bytes": 120 << 30,
                     "loads": [{k: r[k] for k in ("load", "rate", "offered", "accepted", "rejected",
                                                  "completed", "failed", "batches", "throughput",
                                                  "p50_ms", "p99_ms")} for r in served]}
    return out


# ---------------------------------------------------------------------------
# Suite: the other workloads (one JSON line each; not the headline)
# ---------------------------------------------------------------------------

def _timed(fn, stream, reps, flush):
    import torch
    ts = []
    for _ in range(reps):
        flush.fill_(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _run_batch_rate(api, wl, keysets, batch, stream, flush, reps=3, flags=None):
    import torch
    dev = stream.device
    d_in = api.to_device_u64(batch.ct_in, dev)
    d_lut = api.to_device_u32(batch.luts, dev)
    d_out = torch.zeros(batch.out_words, dtype=torch.int64, device=dev)
    keys = [k.ek for k in keysets]
    ws = api.workspace(api.bm_workspace_bytes(keys, batch.jobs), dev)
    if flags is None:
        fn = lambda: api.bm_bootstrap_batch(keys, batch.jobs, d_in, d_lut, d_out, ws, stream)
    else:
        b = api.Batch(keys, batch.jobs, d_in, d_lut, d_out, ws, flags)
        fn = lambda: b.run(stream)
    fn()
    stream.synchronize()
    ms = _timed(fn, stream, reps, flush)
    out = api.from_device_u64(d_out)
    bad = wl.check_outputs(keysets, batch, out)
    return ms, bad, out


def run_suite(args):
    import torch
    from paper_2310_12441_gb300 import api, autotune, serve
    from paper_2310_12441_gb300 import workload as wl
    from paper_2310_12441_gb300.params import JobShape
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    api.load()
    lines = []

    def emit(d):
        d.setdefault("suite", True)
        lines.append(d)
        print(json.dumps(d), flush=True)

    ks1024 = wl.make_keyset(P.KEYS_N1024, 1002)
    # (1) same inputs, m = 4 / N = 1024 versus m = 1 / N = 4096
    if "layouts" in args.suite:
        ks4096 = wl.make_keyset(P.KEYS_N4096, 1002)
        cnt = args.count or 4096
        b4 = wl.make_batch([ks1024], [(0, JobShape(4, 1024), cnt)], 2, interleave=False)
        ms4, bad4, _ = _run_batch_rate(api, wl, [ks1024], b4, stream, flush)
        b1 = wl.make_batch([ks4096], [(0, JobShape(1, 1024), cnt)], 2, interleave=False)
        same = bool(np.array_equal(b1.ct_in, b4.ct_in) and np.array_equal(b1.luts, b4.luts))
        ms1, bad1, _ = _run_batch_rate(api, wl, [ks4096], b1, stream, flush)
        emit({"workload": "same 4096 inputs: BootMMPM m=4 N=1024 vs single polynomial m=1 N=4096",
              "inputs_identical": same,
              "m4_N1024": {"bootstraps_per_s": cnt / ms4 * 1e3, "decrypt_failures": bad4},
              "m1_N4096": {"bootstraps_per_s": cnt / ms1 * 1e3, "decrypt_failures": bad1},
              "speedup_m4_over_m1": ms1 / ms4,
              "key_bytes": {"N1024": ks1024.ek.nbytes, "N4096": ks4096.ek.nbytes}})
        del ks4096
    # (2) large plaintext t = 2^13, m = 8, N = 2048, random / identity tables 50/50
    ks2048 = wl.make_keyset(P.KEYS_N2048, 1003)
    if "large" in args.suite:
        cnt = 2048
        b3 = wl.make_batch([ks2048], [(0, JobShape(8, 8192), cnt)], 3, lut_mix="mixed", interleave=False)
        ms, bad, _ = _run_batch_rate(api, wl, [ks2048], b3, stream, flush)
        emit({"workload": P.LARGE_N2048.name, "bootstraps_per_s": cnt / ms * 1e3, "ms": ms,
              "decrypt_failures": bad, "count": cnt})
    # (3) uneven mix, 8192 jobs over six sets, Zipf(1.2) counts
    if "uneven" in args.suite:
        counts = synth.zipf_counts(8192, len(P.UNEVEN_SETS), 1.2, 5)
        ksets = [ks1024, ks2048]
        groups = [(0 if kp is P.KEYS_N1024 else 1, shape, int(c))
                  for (name, kp, shape), c in zip(P.UNEVEN_SETS, counts)]
        bu = wl.make_batch(ksets, groups, 4)
        d_in = api.to_device_u64(bu.ct_in, dev)
        d_lut = api.to_device_u32(bu.luts, dev)
        d_out = torch.zeros(bu.out_words, dtype=torch.int64, device=dev)
        ws = api.workspace(api.bm_workspace_bytes([k.ek for k in ksets], bu.jobs), dev)
        tuned = autotune.tune(ksets, bu.jobs, d_in, d_lut, d_out, ws, stream, use_cache=False)
        res = {}
        for name, fl in autotune.CANDIDATES.items():
            ms, bad, _ = _run_batch_rate(api, wl, ksets, bu, stream, flush, flags=fl)
            res[name] = {"bootstraps_per_s": len(bu.jobs) / ms * 1e3, "ms": ms, "decrypt_failures": bad}
        emit({"workload": "uneven 8192 jobs, sets S1..S6, Zipf 1.2",
              "counts": {n: int(c) for (n, _, _), c in zip(P.UNEVEN_SETS, counts)},
              "autotune": tuned, "modes": res})
    # (4) served stream over the t = 2^13, m = 8, N = 2048 set
    if "served" in args.suite:
        poolsz = 1024
        bp = wl.make_batch([ks2048], [(0, JobShape(8, 8192), poolsz)], 9, lut_mix="mixed", interleave=False)
        W = P.KEYS_N2048.n + 1
        pool = [(0, 8, 8192, bp.ct_in[i * W:(i + 1) * W], bp.luts[i * 8192:(i + 1) * 8192])
                for i in range(poolsz)]
        cap = None
        for rate in [float(r) for r in args.rates.split(",")]:
            if rate < 1 and cap is not None:
                rate_abs = rate * cap
            else:
                rate_abs = rate
            srv = serve.Server([ks2048], max_batch=args.max_batch, streams=3)
            r = serve.run_open_loop(srv, pool, rate_abs, args.serve_seconds, 11)
            reqs = r.pop("requests")
            if cap is None:
                cap = r["throughput"]
            r["workload"] = "served t=2^13 m=8 N=2048"
            r["capacity_estimate"] = cap
            emit(r)
    # (6) plaintext-size sweep of the Sec. 5 experiments: the identity function
    # (not negacyclic, so two rounds) on log t = 5.., BootMMPM at N = 2^11 with
    # m = 2^(log t - 5), q = 2Nm; the single-polynomial (TFHE) layout where its
    # ring degree N = 2^(log t + 6) is one the library runs (<= 65536)
    if "sweep" in args.suite:
        lo, hi = (int(v) for v in args.sweep_logt.split("-"))
        paper_t1 = {5: 0.7375, 6: 1.3625, 7: 2.6376, 8: 5.2578, 9: 10.203, 10: 20.261, 11: 41.795}
        paper_t1_tfhe = {5: 0.6969, 6: 3.6953, 7: 10.092}

        def key_bytes_formula(kp):
            bsk = 2 * kp.n * 2 * kp.l_B * 2 * kp.N * 8
            ksk = kp.N * kp.l_ks * ((1 << kp.log2_Bks) - 1) * (kp.n + 1) * 8
            return bsk, ksk

        def identity_run(ks, m, logt, count, seed):
            kp = ks.kp
            t = 1 << logt
            T, q = 2 * t, 2 * kp.N * m
            rng = np.random.default_rng(seed)
            x = rng.integers(0, T, count).astype(np.uint32)
            enc = synth.encryption_randomness(kp.n, q, kp.sigma, count, 4000 + seed)
            ct = api.bm_encrypt(ks.sk, q, T, x, enc["mask"], enc["err"])
            f = np.tile(np.arange(t, dtype=np.uint32), count)
            d_in, d_f = api.to_device_u64(ct.ravel(), dev), api.to_device_u32(f, dev)
            d_out = torch.zeros(count * (kp.n + 1), dtype=torch.int64, device=dev)
            ws = api.workspace(api.bm_arbitrary_workspace_bytes(ks.ek, m, t, count), dev)
            run = lambda c: api.bm_bootstrap_arbitrary(ks.ek, m, t, q, d_f, c, d_in, d_out, ws, stream)
            run(1)                                       # warm: one ciphertext
            stream.synchronize()
            plain_ms = _timed(lambda: run(1), stream, 1, flush)
            ms = _timed(lambda: run(count), stream, 1, flush)
            assert api.bm_workspace_status(ws, stream) == 0
            out = api.from_device_u64(d_out).reshape(count, kp.n + 1)
            bad = int(np.sum(api.bm_decrypt(ks.sk, q, T, out) != x % t))
            del ws, d_in, d_f, d_out
            torch.cuda.empty_cache()
            return {"identity_per_s": count / ms * 1e3, "bootstraps_per_s": 2 * count / ms * 1e3,
                    "batch_ms": ms, "count": count, "plain_identity_ms": plain_ms, "decrypt_failures": bad}

        kp_s = P.KEYS_SWEEP_N2048 if args.sweep_n == 512 else \
            P.KeyParams(**{**P.KEYS_SWEEP_N2048.__dict__, "n": args.sweep_n})
        kss = wl.make_keyset(kp_s, 1006)
        for logt in range(lo, hi + 1):
            r = logt - 5
            m = 1 << r
            count = 152 * max(1, 8 >> r)
            res = identity_run(kss, m, logt, count, 600 + logt)
            bsk, ksk = key_bytes_formula(kp_s)
            emit({"workload": f"sweep BootMMPM identity n={kp_s.n} N=2048 log t={logt}",
                  "log_t": logt, "log_q": logt + 7, "log_N": 11, "log_r": r, "m": m, **res,
                  "key_bytes": {"bsk": bsk, "ksk": ksk, "resident": kss.ek.nbytes},
                  "paper_table1_s_per_identity_i7": paper_t1.get(logt) if kp_s.n == 512 else None})
        del kss
        for logt in range(lo, hi + 1):
            logN = logt + 6
            kp_t = P.KeyParams(**{**kp_s.__dict__, "N": 1 << logN})
            bsk, ksk = key_bytes_formula(kp_t)
            d = {"workload": f"sweep TFHE layout identity n={kp_s.n} N=2^{logN} log t={logt}",
                 "log_t": logt, "log_q": logt + 7, "log_N": logN, "m": 1,
                 "key_bytes": {"bsk": bsk, "ksk": ksk},
                 "paper_table1_s_per_identity_i7": paper_t1_tfhe.get(logt) if kp_s.n == 512 else None}
            if logN <= 16:
                kst = wl.make_keyset(kp_t, 1006)
                d.update(identity_run(kst, 1, logt, 152 * max(1, 8 >> (logN - 11)), 700 + logt))
                d["key_bytes"]["resident"] = kst.ek.nbytes
                del kst
                torch.cuda.empty_cache()
            else:
                d["not_run"] = "ring degree above 65536"
            emit(d)
    # (5) decryption failures over >= 1e5 bootstraps of the headline workload
    if "failures" in args.suite:
        total, bad_total = 0, 0
        cnt = 4096
        it = 0
        while total < args.fail_count:
            b = wl.make_batch([ks1024], [(0, JobShape(4, 1024), cnt)], 500 + it, interleave=False)
            _, bad, _ = _run_batch_rate(api, wl, [ks1024], b, stream, flush, reps=1)
            total += cnt
            bad_total += bad
            it += 1
        emit({"workload": P.BATCH_N1024.name, "bootstraps": total, "decrypt_failures": bad_total})
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=P.BATCH_N1024.name, choices=sorted(P.WORKLOADS))
    ap.add_argument("--count", type=int, default=0, help="override the batch size")
    ap.add_argument("--plain", type=int, default=64, help="ciphertexts timed in the plain form")
    ap.add_argument("--cpu-steps", type=int, default=16,
                    help="CMux steps per ciphertext in the bounded oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only (no other workloads, served latency)")
    ap.add_argument("--suite", default="", help="comma list: layouts,large,uneven,served,failures,sweep")
    ap.add_argument("--sweep-logt", default="5-15", help="sweep: range of log2 t")
    ap.add_argument("--sweep-n", type=int, default=512, help="sweep: LWE dimension (512 or 1024)")
    ap.add_argument("--rates", default="2000,0.25,0.5,0.9", help="served: req/s, or fractions of capacity")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--max-batch", type=int, default=512)
    ap.add_argument("--fail-count", type=int, default=100000)
    args = ap.parse_args()
    w = P.WORKLOADS[args.workload]
    if args.suite:
        run_suite(args)
        return
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
