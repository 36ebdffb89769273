"""The no-allocation bootstrap entry point agrees with bm_bootstrap_batch.

bm_bootstrap_batch_noalloc serves callers that cannot allocate device memory
(for example code running inside another application's memory pool, or a
serving loop where cudaMalloc would stall the device): its scratch is a fixed
array inside the library.  This file is collected last so that, if it fails,
a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_workspace_path_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api
    api.load()
    kp = P.KEYS_N1024
    rnd = synth.key_randomness(kp, 1002)
    sk, ek = api.bm_keygen(kp, rnd, 0)
    del rnd
    W = kp.n + 1
    outs = []
    for call, (m, t, cnt) in enumerate([(4, 1024, 24), (2, 512, 40)]):
        qp = 2 * kp.N * m
        msg = synth.messages(t, cnt, 3100 + call)
        enc = synth.encryption_randomness(kp.n, qp, kp.sigma, cnt, 4100 + call)
        ct = api.bm_encrypt(sk, qp, t, msg, enc["mask"], enc["err"])
        luts, _ = synth.luts(t, cnt, 2100 + call)
        jobs = api.make_jobs(0, m, t, np.arange(cnt) * W, np.arange(cnt) * t, np.arange(cnt) * W)
        assert api.bm_workspace_bytes([ek], jobs) <= api.NOALLOC_SCRATCH_BYTES
        d_in = api.to_device_u64(ct.ravel())
        d_lut = api.to_device_u32(luts.ravel())
        ref = torch.zeros(cnt * W, dtype=torch.int64, device="cuda")
        ws = api.workspace(api.bm_workspace_bytes([ek], jobs))
        api.bm_bootstrap_batch([ek], jobs, d_in, d_lut, ref, ws)
        got = torch.full((cnt * W,), -1, dtype=torch.int64, device="cuda")
        status = torch.full((1,), 123, dtype=torch.int32, device="cuda")
        api.bm_bootstrap_batch_noalloc([ek], jobs, d_in, d_lut, got, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert api.bm_workspace_status(ws) == 0
        a, b = api.from_device_u64(ref), api.from_device_u64(got)
        assert np.array_equal(a, b), f"call {call}"
        dec_in = api.bm_decrypt(sk, qp, t, ct)
        dec_out = api.bm_decrypt(sk, kp.Q, t, b.reshape(cnt, W))
        assert np.array_equal(dec_out, luts[np.arange(cnt), dec_in])
        outs.append(b)
    assert outs[0].shape != outs[1].shape or not np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_batches_beyond_the_builtin_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api
    api.load()
    kp = P.KEYS_TOY
    rnd = synth.key_randomness(kp, 1001)
    sk, ek = api.bm_keygen(kp, rnd, 0)
    m, t = 2, 32
    per_job = 2 * 2 * m * kp.N * 8
    cnt = api.NOALLOC_SCRATCH_BYTES // per_job + 8
    jobs = api.make_jobs(0, m, t, 0, 0, 0)
    jobs = np.repeat(jobs, cnt)
    assert api.bm_workspace_bytes([ek], jobs) > api.NOALLOC_SCRATCH_BYTES
    d = torch.zeros(kp.n + 1, dtype=torch.int64, device="cuda")
    dl = torch.zeros(t, dtype=torch.int32, device="cuda")
    with pytest.raises(api.BMError) as e:
        api.bm_bootstrap_batch_noalloc([ek], jobs, d, dl, d)
    assert e.value.code == -8
