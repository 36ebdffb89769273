"""Continuously batched bootstrapping server on one GPU.

Keys stay resident.  Requests (one ciphertext, its table, shape and key set)
enter a bounded host queue; admission also checks a device-memory budget for
keys plus the buffers of everything admitted and not yet finished.  A
scheduler keeps up to `streams` batches in flight, one per CUDA stream: as
soon as a stream is free it takes every queued request (up to `max_batch`)
and launches them as one batch through the C ABI (bm_bootstrap_batch), with
the host-to-device copies, the kernels and the device-to-host copy of the
results on that stream.  A completion thread per stream waits for its batch
and timestamps every request, so requests that arrive while others run are
admitted as soon as a stream frees up and their work overlaps on the device.

Latency of a request = completion time - arrival time (the scheduled Poisson
arrival, so a late producer does not hide queueing).

Failures: tables are checked for negacyclicity at admission (refused with
BM_ENONNEGACYCLIC).  After every batch the completion thread reads (and
clears) the workspace status word; if the device reported an error, each
request of that batch is run again alone on the same stream and only the
ones that fail again are marked failed, with the device's code.

Memory: the per-stream buffers are sized up front for `max_batch` requests
of the largest shape admitted (rows up to `max_m`, tables up to 2 N max_m
entries), and that reservation counts against the memory cap with the keys.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import api
from .workload import KeySet

BM_EBUSY = -7
BM_ENONNEGACYCLIC = -4


@dataclass
class Request:
    rid: int
    key: int
    m: int
    t: int
    ct: np.ndarray          # uint64 [n + 1]
    lut: np.ndarray         # uint32 [t]
    arrival: float
    done: float = 0.0
    out: np.ndarray | None = None
    status: int = 0         # 0, or the device's error code for this request


@dataclass
class Stats:
    accepted: int = 0
    rejected: int = 0
    completed: int = 0
    failed: int = 0
    batches: int = 0
    latencies: list = field(default_factory=list)


class Server:
    def __init__(self, keysets: list[KeySet], max_batch: int = 512, streams: int = 3,
                 queue_cap: int = 2048, mem_cap_bytes: int = 120 << 30, device: int = 0,
                 keep_outputs: bool = False, max_m: int = 8, validate_tables: bool = True):
        import torch
        self.torch = torch
        self.keysets = keysets
        self.keys = [k.ek for k in keysets]
        self.max_batch = max_batch
        self.queue_cap = queue_cap
        self.mem_cap = mem_cap_bytes
        self.keep_outputs = keep_outputs
        self.max_m = max_m
        self.validate_tables = validate_tables
        self.dev = torch.device("cuda", device)
        self.key_bytes = sum(k.nbytes for k in self.keys)
        # per-stream buffers for max_batch requests of the largest shape
        worst = max(self._bytes(ks.kp, max_m, 2 * ks.kp.N * max_m) for ks in keysets)
        self.slab_bytes = int(1.25 * streams * max_batch * worst)   # buffers grow by 1.25x steps
        self.q: collections.deque[Request] = collections.deque()
        self.lock = threading.Condition()
        self.inflight_bytes = 0
        self.stats = Stats()
        self.stop = False
        # per-stream slabs sized for max_batch jobs of the largest shape
        nmax = max(k.kp.n for k in keysets)
        self.slabs = []
        for _ in range(streams):
            self.slabs.append({"stream": torch.cuda.Stream(self.dev), "busy": False,
                               "in": None, "lut": None, "out": None, "ws": None,
                               "h_in": None, "h_lut": None, "h_out": None, "nmax": nmax})
        self.threads = []

    # -- admission -------------------------------------------------------------------
    @staticmethod
    def _bytes(kp, m: int, t: int) -> int:
        """Device bytes of one request: input and output ciphertext, table,
        and the three [m][2][N] accumulator buffers of its workspace."""
        return 2 * (kp.n + 1) * 8 + t * 4 + 3 * 2 * m * kp.N * 8 + 64

    def request_bytes(self, r: Request) -> int:
        return self._bytes(self.keysets[r.key].kp, r.m, r.t)

    def submit(self, r: Request) -> int:
        """Admits a request (0) or refuses it (BM_EBUSY; BM_ENONNEGACYCLIC
        for a table that is not negacyclic when tables are validated)."""
        if r.m > self.max_m:
            return BM_EBUSY
        if self.validate_tables:
            lut = np.asarray(r.lut, dtype=np.int64)
            h = r.t // 2
            if lut.size != r.t or (lut >= r.t).any() or \
                    not np.array_equal(lut[h:], (r.t - lut[:h]) % r.t):
                with self.lock:
                    self.stats.rejected += 1
                return BM_ENONNEGACYCLIC
        nb = self.request_bytes(r)
        with self.lock:
            if len(self.q) >= self.queue_cap or \
                    self.key_bytes + self.slab_bytes + self.inflight_bytes + nb > self.mem_cap:
                self.stats.rejected += 1
                return BM_EBUSY
            self.inflight_bytes += nb
            self.q.append(r)
            self.stats.accepted += 1
            self.lock.notify_all()
        return 0

    # -- device side ----------------------------------------------------------------------
    def _ensure(self, slab, words_in, words_lut, words_out, ws_bytes):
        torch = self.torch
        def grow(name, n, dtype, pinned=False):
            cur = slab[name]
            if cur is None or cur.numel() < n:
                n2 = max(n, int(1.25 * (cur.numel() if cur is not None else 0)))
                if pinned:
                    slab[name] = torch.empty(n2, dtype=dtype).pin_memory()
                elif name == "ws":
                    # the workspace's status word must start at zero
                    slab[name] = torch.zeros(n2, dtype=dtype, device=self.dev)
                else:
                    slab[name] = torch.empty(n2, dtype=dtype, device=self.dev)
        grow("in", words_in, torch.int64)
        grow("lut", words_lut, torch.int32)
        grow("out", words_out, torch.int64)
        grow("ws", ws_bytes, torch.uint8)
        grow("h_in", words_in, torch.int64, True)
        grow("h_lut", words_lut, torch.int32, True)
        grow("h_out", words_out, torch.int64, True)

    def _launch(self, slab, reqs: list[Request]):
        torch = self.torch
        jobs = np.zeros(len(reqs), api.JOB_DTYPE)
        in_off = lut_off = 0
        for j, r in enumerate(reqs):
            n = self.keysets[r.key].kp.n
            jobs[j] = (r.key, r.m, r.t, 0, in_off, lut_off, in_off)
            in_off += n + 1
            lut_off += r.t
        ws_bytes = api.bm_workspace_bytes(self.keys, jobs)
        self._ensure(slab, in_off, lut_off, in_off, ws_bytes)
        h_in = slab["h_in"].numpy().view(np.uint64)
        h_lut = slab["h_lut"].numpy().view(np.uint32)
        for j, r in enumerate(reqs):
            o, lo = int(jobs[j]["in_off"]), int(jobs[j]["lut_off"])
            h_in[o:o + r.ct.size] = r.ct
            h_lut[lo:lo + r.t] = r.lut
        st = slab["stream"]
        with torch.cuda.stream(st):
            slab["in"][:in_off].copy_(slab["h_in"][:in_off], non_blocking=True)
            slab["lut"][:lut_off].copy_(slab["h_lut"][:lut_off], non_blocking=True)
            api.bm_bootstrap_batch(self.keys, jobs, slab["in"], slab["lut"], slab["out"], slab["ws"], st)
            slab["h_out"][:in_off].copy_(slab["out"][:in_off], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return jobs, ev

    def _isolate(self, slab, reqs: list[Request], code: int):
        """The device reported `code` for a batch: run each request alone on
        the slab's stream and mark those that fail again."""
        for r in reqs:
            _, ev = self._launch(slab, [r])
            ev.synchronize()
            c = api.bm_workspace_status(slab["ws"], slab["stream"])
            r.status = c
            if c == 0 and self.keep_outputs:
                r.out = slab["h_out"].numpy().view(np.uint64)[:r.ct.size].copy()

    def _complete(self, slab, reqs, jobs, ev):
        ev.synchronize()
        code = api.bm_workspace_status(slab["ws"], slab["stream"])   # reads and clears
        now = time.perf_counter()
        out = slab["h_out"].numpy().view(np.uint64)
        nb = 0
        for j, r in enumerate(reqs):
            r.done = now
            if self.keep_outputs:
                o = int(jobs[j]["out_off"])
                r.out = out[o:o + r.ct.size].copy()
            nb += self.request_bytes(r)
        if code != 0:
            self._isolate(slab, reqs, code)
        failed = sum(1 for r in reqs if r.status != 0)
        with self.lock:
            self.inflight_bytes -= nb
            self.stats.completed += len(reqs) - failed
            self.stats.failed += failed
            self.stats.latencies.extend(r.done - r.arrival for r in reqs if r.status == 0)
            slab["busy"] = False
            self.lock.notify_all()

    def _scheduler(self):
        while True:
            with self.lock:
                while not self.stop and (not self.q or all(s["busy"] for s in self.slabs)):
                    self.lock.wait(0.05)
                if self.stop and not self.q:
                    return
                free = [s for s in self.slabs if not s["busy"]]
                if not free or not self.q:
                    self.lock.wait(0.05)
                    continue
                slab = free[0]
                take = min(len(self.q), self.max_batch)
                reqs = [self.q.popleft() for _ in range(take)]
                slab["busy"] = True
                self.stats.batches += 1
            jobs, ev = self._launch(slab, reqs)
            th = threading.Thread(target=self._complete, args=(slab, reqs, jobs, ev), daemon=True)
            th.start()
            self.threads.append(th)

    def start(self):
        self.sched = threading.Thread(target=self._scheduler, daemon=True)
        self.sched.start()

    def drain_and_stop(self, timeout: float = 600.0):
        t0 = time.perf_counter()
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        self.sched.join(timeout)
        for th in self.threads:
            th.join(max(0.0, timeout - (time.perf_counter() - t0)))


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    return t[t < duration]


def run_open_loop(server: Server, pool: list[tuple[int, int, int, np.ndarray, np.ndarray]],
                  rate: float, duration: float, seed: int) -> dict:
    """Drives the server with Poisson arrivals at `rate` for `duration` seconds
    (requests cycle through `pool`), then waits for every admitted request."""
    arr = poisson_arrivals(rate, duration, seed)
    server.start()
    t0 = time.perf_counter()
    reqs = []
    for i, ta in enumerate(arr):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        key, m, t, ct, lut = pool[i % len(pool)]
        r = Request(i, key, m, t, ct, lut, t0 + ta)
        if server.submit(r) == 0:
            reqs.append(r)
    offered_end = time.perf_counter()
    server.drain_and_stop()
    end = time.perf_counter()
    lat = np.array(server.stats.latencies) if server.stats.latencies else np.array([np.nan])
    return {"rate": rate, "duration_s": duration, "offered": int(len(arr)),
            "accepted": server.stats.accepted, "rejected": server.stats.rejected,
            "completed": server.stats.completed, "failed": server.stats.failed,
            "batches": server.stats.batches,
            "throughput": server.stats.completed / (end - t0),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "drain_s": end - offered_end, "requests": reqs}
