"""Full-length parity on the production key sets: every CMux step of
Algorithm 1 runs with a nonzero mask entry in general (no prefix
ciphertexts), and the GPU output equals the oracle's word for word.

Expected outputs come from tests/golden/full_length_*.json, written by
tests/golden/make_full_length.py, which calls only the oracle (all n steps
take minutes per ciphertext on the CPU).  The GPU side regenerates keys and
ciphertexts from the stored seeds with the library's own seeded entry points
(bm_keygen_seeded on the device, bm_encrypt_seeded), checks that the
ciphertexts hash to the oracle's, and bootstraps them through the C ABI in
each launch form: thread-block clusters (rows split), one block per job, the
persistent kernel and a replayed CUDA graph.  One headline-set ciphertext is
also bootstrapped by the oracle live, at full length, in this run.
"""
import glob
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
KEYS = {"n630_N1024": P.KEYS_N1024, "n630_N4096": P.KEYS_N4096, "n750_N2048": P.KEYS_N2048}


def golden(case):
    with open(os.path.join(GOLD, f"full_length_{case}.json")) as f:
        return json.load(f)


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _words(hexrow):
    return np.array([int(hexrow[i:i + 16], 16) for i in range(0, len(hexrow), 16)], dtype=np.uint64)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


_keys = {}


def keyset(api, name, seed):
    if (name, seed) not in _keys:
        _keys[(name, seed)] = api.bm_keygen_seeded(KEYS[name], seed)
    return _keys[(name, seed)]


def case_inputs(api, g):
    """Keys, ciphertexts, tables and expected outputs of a golden case."""
    sk, ek = keyset(api, g["key_set"], g["key_seed"])
    kp = KEYS[g["key_set"]]
    assert g["params"]["Q"] == kp.Q and g["params"]["n"] == kp.n and g["params"]["N"] == kp.N
    t, cnt = g["t"], g["count"]
    luts, ident = synth.luts(t, cnt, g["lut_seed"], mix=g["lut_mix"])
    msg = synth.messages(t, cnt, g["msg_seed"], half=ident)
    assert _sha(luts) == g["lut_sha256"], "the seeded input generator's stream differs on this platform"
    assert [int(x) for x in msg] == g["messages"]
    ct = api.bm_encrypt_seeded(sk, g["q_prime"], t, msg, g["enc_seed"])
    assert _sha(ct) == g["ct_sha256"], "library seeded encryption differs from the oracle's"
    assert int((ct[:, :kp.n] != 0).sum()) == g["nonzero_mask_entries"] >= cnt * kp.n * 0.99
    want = np.stack([_words(r) for r in g["out"]])
    return sk, ek, kp, ct, luts, want


def _run(api, keys, jobs, ct_flat, luts_flat, out_words, flags=None, stream=None):
    d_in = api.to_device_u64(ct_flat)
    d_lut = api.to_device_u32(luts_flat)
    d_out = torch.zeros(out_words, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes(keys, jobs))
    if flags is None:
        api.bm_bootstrap_batch(keys, jobs, d_in, d_lut, d_out, ws)
    else:
        b = api.Batch(keys, jobs, d_in, d_lut, d_out, ws, flags)
        s = stream or torch.cuda.current_stream()
        for _ in range(2 if flags & api.BATCH_GRAPH else 1):     # capture, then replay
            d_out.zero_()
            b.run(s)
            s.synchronize()
        b.free()
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    return api.from_device_u64(d_out)


def _uniform_jobs(api, count, n, t, m):
    W = n + 1
    return api.make_jobs(0, m, t, np.arange(count) * W, np.arange(count) * t, np.arange(count) * W)


def test_golden_files_are_complete():
    names = sorted(os.path.basename(p) for p in glob.glob(os.path.join(GOLD, "full_length_*.json")))
    assert len(names) == 9, names


@pytest.mark.parametrize("form", ["cluster", "one_block", "persistent_graph"])
def test_full_length_n630_N1024_m4(api, form):
    g = golden("n630_N1024_m4")
    sk, ek, kp, ct, luts, want = case_inputs(api, g)
    jobs = _uniform_jobs(api, g["count"], kp.n, g["t"], g["m"])
    flags = {"cluster": None, "one_block": api.BATCH_ONE_BLOCK,
             "persistent_graph": api.BATCH_PERSISTENT | api.BATCH_GRAPH}[form]
    stream = torch.cuda.Stream() if form == "persistent_graph" else None
    got = _run(api, [ek], jobs, ct.ravel(), luts.ravel(), ct.size, flags, stream)
    assert np.array_equal(got.reshape(want.shape), want)


def test_full_length_n630_N4096_m1_same_inputs(api):
    """The single-polynomial layout bootstraps the very same ciphertexts
    (same seed, same s, q' = 8192) and matches its own oracle outputs."""
    g = golden("n630_N4096_m1")
    sk, ek, kp, ct, luts, want = case_inputs(api, g)
    assert g["ct_sha256"] == golden("n630_N1024_m4")["ct_sha256"]
    jobs = _uniform_jobs(api, g["count"], kp.n, g["t"], g["m"])
    for flags in (None, api.BATCH_ONE_BLOCK):
        got = _run(api, [ek], jobs, ct.ravel(), luts.ravel(), ct.size, flags)
        assert np.array_equal(got.reshape(want.shape), want)


def test_full_length_n750_N2048_m8_random_and_identity(api):
    g = golden("n750_N2048_m8")
    assert g["lut_mix"] == "mixed"            # job 0 random table, job 1 identity refresh
    sk, ek, kp, ct, luts, want = case_inputs(api, g)
    assert np.array_equal(luts[1][: g["t"] // 2], np.arange(g["t"] // 2))
    jobs = _uniform_jobs(api, g["count"], kp.n, g["t"], g["m"])
    for flags in (None, api.BATCH_ONE_BLOCK):
        got = _run(api, [ek], jobs, ct.ravel(), luts.ravel(), ct.size, flags)
        assert np.array_equal(got.reshape(want.shape), want)


@pytest.mark.parametrize("flags", ["persistent", "grouped_graph"])
def test_full_length_uneven_sets_in_one_launch(api, flags):
    """One ciphertext of each of the six parameter sets of the uneven batch
    (two key sets, m = 1..8, N = 1024 / 2048) in one launch."""
    cases = [golden(f"uneven_S{i}") for i in range(1, 7)]
    keys, key_idx, cts, lts, wants, jobs = [], {}, [], [], [], []
    in_off = lut_off = 0
    for g in cases:
        sk, ek, kp, ct, luts, want = case_inputs(api, g)
        k = g["key_set"]
        if k not in key_idx:
            key_idx[k] = len(keys)
            keys.append(ek)
        jobs.append((key_idx[k], g["m"], g["t"], 0, in_off, lut_off, in_off))
        cts.append(ct[0])
        lts.append(luts[0])
        wants.append(want[0])
        in_off += kp.n + 1
        lut_off += g["t"]
    jobs = np.array(jobs, dtype=api.JOB_DTYPE)
    fl = api.BATCH_PERSISTENT if flags == "persistent" else api.BATCH_GRAPH
    stream = torch.cuda.Stream()
    got = _run(api, keys, jobs, np.concatenate(cts), np.concatenate(lts), in_off, fl, stream)
    for j, w in zip(jobs, wants):
        o = int(j["out_off"])
        assert np.array_equal(got[o:o + len(w)], w), j


def test_full_length_live_oracle_n630_N1024(api, orc):
    """One headline-set ciphertext with all 630 CMux steps, bootstrapped by the
    oracle in this run (keys from the oracle's own seeded streams) and on the
    GPU (keys drawn on the device)."""
    kp, m, t = P.KEYS_N1024, 4, 1024
    seed = 1002
    sk, ek = keyset(api, "n630_N1024", seed)
    rnd = orc.seeded_key_randomness(kp, seed)
    bsk, ksk = orc.keygen_bsk(kp, rnd), orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    msg = synth.messages(t, 1, 3950)
    ct = api.bm_encrypt_seeded(sk, qp, t, msg, 4950)
    assert int((ct[0, :kp.n] != 0).sum()) >= kp.n - 3
    luts, _ = synth.luts(t, 1, 2950)
    got = _run(api, [ek], _uniform_jobs(api, 1, kp.n, t, m), ct.ravel(), luts.ravel(), kp.n + 1)
    want = orc.bootstrap(kp, m, t, bsk, ksk, ct, luts)[0]
    assert np.array_equal(got, want)
