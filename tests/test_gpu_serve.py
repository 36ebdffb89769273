"""The continuously batched server returns, for every request, exactly the
ciphertext that bootstrapping the same request alone returns (tolerance 0:
all arithmetic is exact), and refuses requests beyond its admission limits."""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api, serve
    from paper_2310_12441_gb300 import workload as wl
    api.load()
    ksets = [wl.make_keyset(P.KEYS_TOY, 1001), wl.make_keyset(P.KEYS_N1024, 1002)]
    return api, serve, wl, ksets


def _pool(wl, ksets):
    from paper_2310_12441_gb300.params import JobShape
    b = wl.make_batch(ksets, [(0, JobShape(2, 32), 6), (1, JobShape(4, 1024), 5),
                              (1, JobShape(1, 256), 5), (1, JobShape(2, 512), 4)], 77)
    pool = []
    for j in b.jobs:
        n = ksets[int(j["key"])].kp.n
        o, lo = int(j["in_off"]), int(j["lut_off"])
        pool.append((int(j["key"]), int(j["m"]), int(j["t"]), b.ct_in[o:o + n + 1].copy(),
                     b.luts[lo:lo + int(j["t"])].copy()))
    return pool


def test_served_results_equal_results_alone(env):
    api, serve, wl, ksets = env
    pool = _pool(wl, ksets)
    srv = serve.Server(ksets, max_batch=7, streams=3, keep_outputs=True)
    r = serve.run_open_loop(srv, pool, rate=60.0, duration=1.5, seed=3)
    reqs = r["requests"]
    assert r["rejected"] == 0 and r["completed"] == len(reqs) > 20
    assert r["batches"] > 1
    keys = [k.ek for k in ksets]
    for req in reqs[:len(pool)]:
        n = ksets[req.key].kp.n
        job = api.make_jobs(req.key, req.m, req.t, 0, 0, 0)
        d_out = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        ws = api.workspace(api.bm_workspace_bytes(keys, job))
        api.bm_bootstrap_batch(keys, job, api.to_device_u64(req.ct), api.to_device_u32(req.lut), d_out, ws)
        torch.cuda.synchronize()
        assert np.array_equal(api.from_device_u64(d_out), req.out), req.rid


def test_admission_refuses_beyond_limits(env):
    api, serve, wl, ksets = env
    pool = _pool(wl, ksets)
    srv = serve.Server(ksets, max_batch=4, streams=1, queue_cap=3)
    reqs = [serve.Request(i, *pool[i % len(pool)], arrival=0.0) for i in range(8)]
    codes = [srv.submit(r) for r in reqs]          # scheduler not started: queue fills
    assert codes[:3] == [0, 0, 0] and all(c == serve.BM_EBUSY for c in codes[3:])
    small = serve.Server(ksets, mem_cap_bytes=sum(k.ek.nbytes for k in ksets) + 1)
    assert small.submit(serve.Request(0, *pool[0], arrival=0.0)) == serve.BM_EBUSY
    # the stream buffers' reservation counts against the cap too
    roomy = serve.Server(ksets, max_batch=4, streams=1)
    tight = serve.Server(ksets, max_batch=4, streams=1,
                         mem_cap_bytes=roomy.key_bytes + roomy.slab_bytes // 2)
    assert roomy.submit(serve.Request(0, *pool[0], arrival=0.0)) == 0
    assert tight.submit(serve.Request(0, *pool[0], arrival=0.0)) == serve.BM_EBUSY


def test_device_error_is_reported_for_the_bad_request_only(env):
    """A table that is not negacyclic, let through admission, makes the device
    set the workspace status word; the server reads it, re-runs the batch's
    requests alone, and fails only the bad one (BM_ENONNEGACYCLIC).  With table
    validation on, admission refuses it."""
    api, serve, wl, ksets = env
    pool = _pool(wl, ksets)[:6]
    key, m, t, ct, lut = pool[2]
    bad_lut = lut.copy()
    bad_lut[t // 2] = (bad_lut[t // 2] + 1) % t
    pool[2] = (key, m, t, ct, bad_lut)
    srv = serve.Server(ksets, max_batch=8, streams=1, keep_outputs=True, validate_tables=False)
    reqs = [serve.Request(i, *pool[i], arrival=0.0) for i in range(len(pool))]
    assert all(srv.submit(r) == 0 for r in reqs)       # queued before the scheduler starts
    srv.start()
    srv.drain_and_stop()
    assert srv.stats.batches == 1
    assert [r.status for r in reqs] == [0, 0, serve.BM_ENONNEGACYCLIC, 0, 0, 0]
    assert srv.stats.failed == 1 and srv.stats.completed == 5
    keys = [k.ek for k in ksets]
    for r in reqs:
        if r.status:
            continue
        n = ksets[r.key].kp.n
        job = api.make_jobs(r.key, r.m, r.t, 0, 0, 0)
        d_out = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        ws = api.workspace(api.bm_workspace_bytes(keys, job))
        api.bm_bootstrap_batch(keys, job, api.to_device_u64(r.ct), api.to_device_u32(r.lut), d_out, ws)
        torch.cuda.synchronize()
        assert np.array_equal(api.from_device_u64(d_out), r.out), r.rid
    strict = serve.Server(ksets, max_batch=8, streams=1)
    assert strict.submit(serve.Request(9, *pool[2], arrival=0.0)) == serve.BM_ENONNEGACYCLIC
