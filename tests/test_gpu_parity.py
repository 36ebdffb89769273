"""Parity of the CUDA path with the oracle, element by element, bit-exact.

All arithmetic is exact modular integer arithmetic, so the tolerance is 0:
every output word must equal the oracle's.  Every call goes through the C ABI
(libbootmmpm.so) via the thin binding.
"""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    return A


class KeySet:
    def __init__(self, api, orc, kp, seed, oracle_keys):
        self.kp = kp
        self.rnd = synth.key_randomness(kp, seed)
        self.sk, self.ek = api.bm_keygen(kp, self.rnd, 0)
        self.bsk = orc.keygen_bsk(kp, self.rnd, 0, oracle_keys)
        self.ksk = orc.keygen_ksk(kp, self.rnd)


@pytest.fixture(scope="module")
def toy(api, orc):
    return KeySet(api, orc, P.KEYS_TOY, 1001, P.KEYS_TOY.n)


@pytest.fixture(scope="module")
def n1024(api, orc):
    return KeySet(api, orc, P.KEYS_N1024, 1002, 8)


@pytest.fixture(scope="module")
def n2048(api, orc):
    return KeySet(api, orc, P.KEYS_N2048, 1003, 4)


@pytest.fixture(scope="module")
def n4096(api, orc):
    return KeySet(api, orc, P.KEYS_N4096, 1002, 3)


def _encrypt(orc, ks, m, t, count, seed, prefix=None, half=None):
    kp = ks.kp
    qp = 2 * kp.N * m
    msg = synth.messages(t, count, 3000 + seed, half)
    enc = synth.encryption_randomness(kp.n, qp, kp.sigma, count, 4000 + seed, prefix=prefix)
    ct = orc.encrypt(kp.n, qp, t, ks.rnd["s"], msg, enc["mask"], enc["err"])
    return msg, ct


def _run_batch(api, keys, jobs, ct_in, luts, out_words):
    d_in = api.to_device_u64(ct_in.ravel())
    d_lut = api.to_device_u32(luts.ravel())
    d_out = torch.zeros(out_words, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes(keys, jobs))
    api.bm_bootstrap_batch(keys, jobs, d_in, d_lut, d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    return api.from_device_u64(d_out)


def _uniform_jobs(api, count, n, t, m):
    return api.make_jobs(0, m, t, np.arange(count) * (n + 1), np.arange(count) * t,
                         np.arange(count) * (n + 1))


# --- ring product (NTT / INTT path) --------------------------------------------------

@pytest.mark.parametrize("fixture", ["toy", "n1024", "n2048"])
def test_poly_mul_matches_schoolbook(api, orc, request, fixture):
    ks = request.getfixturevalue(fixture)
    kp = ks.kp
    rng = np.random.default_rng(kp.N)
    cnt = 3
    a = rng.integers(0, kp.Q, (cnt, kp.N), dtype=np.uint64)
    b = rng.integers(0, kp.Q, (cnt, kp.N), dtype=np.uint64)
    a[0] = 0; a[0, 1] = 1                      # x * b
    b[1] = kp.Q - 1                            # all coefficients -1
    d_out = torch.zeros(cnt * kp.N, dtype=torch.int64, device="cuda")
    api.bm_poly_mul(ks.ek, api.to_device_u64(a), api.to_device_u64(b), cnt, d_out)
    got = api.from_device_u64(d_out).reshape(cnt, kp.N)
    for i in range(cnt):
        assert np.array_equal(got[i], orc.poly_mul(kp.N, kp.Q, a[i], b[i])), i


# --- sample extraction and key switching -----------------------------------------------

@pytest.mark.parametrize("fixture", ["toy", "n1024"])
def test_sample_extract(api, orc, request, fixture):
    ks = request.getfixturevalue(fixture)
    kp = ks.kp
    rng = np.random.default_rng(3)
    cnt = 5
    rl = rng.integers(0, kp.Q, (cnt, 2, kp.N), dtype=np.uint64)
    rl[0, 0] = 0                                # zero a-part (no negation wrap)
    d_out = torch.zeros(cnt * (kp.N + 1), dtype=torch.int64, device="cuda")
    api.bm_sample_extract(ks.ek, api.to_device_u64(rl), cnt, d_out)
    got = api.from_device_u64(d_out).reshape(cnt, kp.N + 1)
    for i in range(cnt):
        assert np.array_equal(got[i], orc.sample_extract(kp.N, kp.Q, rl[i, 0], rl[i, 1]))


@pytest.mark.parametrize("fixture", ["toy", "n1024", "n2048"])
def test_key_switch(api, orc, request, fixture):
    ks = request.getfixturevalue(fixture)
    kp = ks.kp
    rng = np.random.default_rng(5)
    cnt = 4
    lwe = rng.integers(0, kp.Q, (cnt, kp.N + 1), dtype=np.uint64)
    lwe[1, :kp.N] = 0                           # all digits zero: output (0, b)
    lwe[2, :kp.N] = kp.Q - 1                    # rounding to P wraps to 0
    d_out = torch.zeros(cnt * (kp.n + 1), dtype=torch.int64, device="cuda")
    api.bm_key_switch(ks.ek, api.to_device_u64(lwe), cnt, d_out)
    got = api.from_device_u64(d_out).reshape(cnt, kp.n + 1)
    for i in range(cnt):
        assert np.array_equal(got[i], orc.key_switch(kp, lwe[i], ks.ksk)), i


@pytest.mark.parametrize("cnt", [1, 30, 40, 77, 160])
def test_key_switch_every_cluster_split(api, orc, n1024, cnt):
    """The key switch splits a job over a cluster of S = 8, 4, 2 or 1 blocks,
    the largest S with cnt S <= SMs (152 SMs: 1 -> 8, 30 -> 4, 40 -> 2,
    77 and 160 -> 1); every split gives the oracle's words."""
    kp = n1024.kp
    rng = np.random.default_rng(cnt)
    lwe = rng.integers(0, kp.Q, (cnt, kp.N + 1), dtype=np.uint64)
    d_out = torch.zeros(cnt * (kp.n + 1), dtype=torch.int64, device="cuda")
    api.bm_key_switch(n1024.ek, api.to_device_u64(lwe), cnt, d_out)
    got = api.from_device_u64(d_out).reshape(cnt, kp.n + 1)
    for i in sorted({0, cnt // 2, cnt - 1}):
        assert np.array_equal(got[i], orc.key_switch(kp, lwe[i], n1024.ksk)), (cnt, i)


# --- blind rotation ----------------------------------------------------------------------

def _blind_rotate_gpu(api, ks, jobs, ct, luts, steps):
    kp = ks.kp
    out_words = int(sum(2 * int(j["m"]) * kp.N for j in jobs))
    jobs = jobs.copy()
    offs = np.concatenate([[0], np.cumsum([2 * int(j["m"]) * kp.N for j in jobs])[:-1]])
    jobs["out_off"] = offs
    d_out = torch.zeros(out_words, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([ks.ek], jobs))
    api.bm_blind_rotate([ks.ek], jobs, steps, api.to_device_u64(ct.ravel()),
                        api.to_device_u32(luts.ravel()), d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    full = api.from_device_u64(d_out)
    return [full[o:o + 2 * int(j["m"]) * kp.N].reshape(int(j["m"]), 2, kp.N) for o, j in zip(offs, jobs)]


def test_blind_rotate_toy_full(api, orc, toy):
    kp, m, t = toy.kp, 2, 32
    msg, ct = _encrypt(orc, toy, m, t, 3, 1)
    luts, _ = synth.luts(t, 3, 2001)
    jobs = _uniform_jobs(api, 3, kp.n, t, m)
    got = _blind_rotate_gpu(api, toy, jobs, ct, luts, 1 << 30)
    for i in range(3):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, toy.bsk, ct[i], luts[i]))


@pytest.mark.parametrize("m,t", [(64, 1 << 12), (1024, 1 << 14)])
def test_blind_rotate_toy_many_rows(api, orc, toy, m, t):
    """Large m (the plaintext-size sweep goes to m = 1024): each of a
    cluster's 8 blocks takes m/8 rows; prefix ciphertexts keep the oracle fast."""
    kp = toy.kp
    _, ct = _encrypt(orc, toy, m, t, 2, 5 + m, prefix=2)
    luts, _ = synth.luts(t, 2, 2005 + m)
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    got = _blind_rotate_gpu(api, toy, jobs, ct, luts, 1 << 30)
    for i in range(2):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, toy.bsk, ct[i], luts[i])), i


@pytest.mark.parametrize("steps", [0, 1, 5])
def test_blind_rotate_steps_equal_truncated_ciphertext(api, orc, n1024, steps):
    """ACC after the first K CMux steps equals the oracle's full rotation of
    the same ciphertext with a_k = 0 beyond K (P(0) = I)."""
    kp, m, t = n1024.kp, 4, 1024
    msg, ct = _encrypt(orc, n1024, m, t, 2, 2)
    luts, _ = synth.luts(t, 2, 2002)
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    got = _blind_rotate_gpu(api, n1024, jobs, ct, luts, steps)
    for i in range(2):
        tr = ct[i].copy()
        tr[steps:kp.n] = 0
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, n1024.bsk, tr, luts[i]))


def test_blind_rotate_prefix_ciphertexts_n2048(api, orc, n2048):
    kp, m, t = n2048.kp, 8, 8192
    msg, ct = _encrypt(orc, n2048, m, t, 2, 3, prefix=4)
    luts, _ = synth.luts(t, 2, 2003, mix="mixed")
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    got = _blind_rotate_gpu(api, n2048, jobs, ct, luts, 1 << 30)
    for i in range(2):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, n2048.bsk, ct[i], luts[i]))


def test_blind_rotate_single_polynomial_n4096(api, orc, n4096):
    """The m = 1, N = 4096 layout (same q' = 8192 and t as the N = 1024, m = 4
    batch), prefix ciphertexts, bit-exact."""
    kp, m, t = n4096.kp, 1, 1024
    msg, ct = _encrypt(orc, n4096, m, t, 2, 4, prefix=3)
    luts, _ = synth.luts(t, 2, 2004)
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    got = _blind_rotate_gpu(api, n4096, jobs, ct, luts, 1 << 30)
    for i in range(2):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, n4096.bsk, ct[i], luts[i]))


def test_bootstrap_prefix_n4096_bit_exact(api, orc, n4096):
    kp, m, t = n4096.kp, 1, 1024
    msg, ct = _encrypt(orc, n4096, m, t, 2, 5, prefix=3)
    luts, _ = synth.luts(t, 2, 2005)
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    got = _run_batch(api, [n4096.ek], jobs, ct, luts, 2 * (kp.n + 1)).reshape(2, kp.n + 1)
    assert np.array_equal(got, orc.bootstrap(kp, m, t, n4096.bsk, n4096.ksk, ct, luts))


@pytest.mark.parametrize("m,t", [(2, 1 << 11), (4, 1 << 12), (1, 1 << 10)])
def test_blind_rotate_n2048_other_shapes(api, orc, n2048, m, t):
    kp = n2048.kp
    msg, ct = _encrypt(orc, n2048, m, t, 3, 6 + m, prefix=4)
    luts, _ = synth.luts(t, 3, 2006 + m)
    jobs = _uniform_jobs(api, 3, kp.n, t, m)
    got = _blind_rotate_gpu(api, n2048, jobs, ct, luts, 1 << 30)
    for i in range(3):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, n2048.bsk, ct[i], luts[i]))


def test_blind_rotate_uneven_shapes_one_call(api, orc, n1024):
    """Jobs with different (m, t) in one call (the uneven-batch sets on the
    N = 1024 key), prefix ciphertexts so the oracle stays fast."""
    kp = n1024.kp
    shapes = [(1, 256), (2, 512), (4, 1024), (2, 512), (1, 256), (3, 768), (5, 1280)]
    cts, luts_l, jobs = [], [], []
    in_off = lut_off = 0
    for i, (m, t) in enumerate(shapes):
        _, ct = _encrypt(orc, n1024, m, t, 1, 10 + i, prefix=6)
        lut, _ = synth.luts(t, 1, 2010 + i)
        cts.append(ct[0]); luts_l.append(lut[0])
        jobs.append((0, m, t, 0, in_off, lut_off, 0))
        in_off += kp.n + 1; lut_off += t
    jobs = np.array(jobs, dtype=api.JOB_DTYPE)
    got = _blind_rotate_gpu(api, n1024, jobs, np.concatenate(cts), np.concatenate(luts_l), 1 << 30)
    for i, (m, t) in enumerate(shapes):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, n1024.bsk, cts[i], luts_l[i])), i


# --- full bootstrap ------------------------------------------------------------------------

def test_bootstrap_toy_all_messages(api, orc, toy):
    """Toy workload: all 32 messages, bit-exact with the oracle, and every
    output decrypts to f(Dec(input))."""
    kp, m, t = toy.kp, 2, 32
    msg = np.arange(t, dtype=np.uint32)
    qp = 2 * kp.N * m
    enc = synth.encryption_randomness(kp.n, qp, kp.sigma, t, 4001)
    ct = orc.encrypt(kp.n, qp, t, toy.rnd["s"], msg, enc["mask"], enc["err"])
    luts, _ = synth.luts(t, t, 2001)
    jobs = _uniform_jobs(api, t, kp.n, t, m)
    got = _run_batch(api, [toy.ek], jobs, ct, luts, t * (kp.n + 1)).reshape(t, kp.n + 1)
    want = orc.bootstrap(kp, m, t, toy.bsk, toy.ksk, ct, luts)
    assert np.array_equal(got, want)
    dec_in = orc.decrypt(kp.n, qp, t, toy.rnd["s"], ct)
    dec_out = api.bm_decrypt(toy.sk, kp.Q, t, got)
    assert np.array_equal(dec_out, luts[np.arange(t), dec_in])


def test_bootstrap_prefix_n1024_bit_exact(api, orc, n1024):
    kp, m, t = n1024.kp, 4, 1024
    cnt = 3
    msg, ct = _encrypt(orc, n1024, m, t, cnt, 21, prefix=8)
    luts, _ = synth.luts(t, cnt, 2021)
    jobs = _uniform_jobs(api, cnt, kp.n, t, m)
    got = _run_batch(api, [n1024.ek], jobs, ct, luts, cnt * (kp.n + 1)).reshape(cnt, kp.n + 1)
    want = orc.bootstrap(kp, m, t, n1024.bsk, n1024.ksk, ct, luts)
    assert np.array_equal(got, want)


def test_nonnegacyclic_table_sets_status(api, orc, toy):
    kp, m, t = toy.kp, 2, 32
    _, ct = _encrypt(orc, toy, m, t, 2, 30)
    luts, _ = synth.luts(t, 2, 2030)
    luts[1, t // 2] = (luts[1, t // 2] + 1) % t
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    d_out = torch.zeros(2 * (kp.n + 1), dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([toy.ek], jobs))
    api.bm_bootstrap_batch([toy.ek], jobs, api.to_device_u64(ct.ravel()),
                           api.to_device_u32(luts.ravel()), d_out, ws)
    assert api.bm_workspace_status(ws) == -4
    assert api.bm_workspace_status(ws) == 0          # reading clears it


def test_invalid_jobs_rejected_before_launch(api, toy):
    kp = toy.kp
    ws = api.workspace(1 << 20)
    d = torch.zeros(64, dtype=torch.int64, device="cuda")
    for bad in [dict(m=0), dict(t=3), dict(t=2 * kp.N * 2 + 2), dict(key=1)]:
        j = api.make_jobs(bad.get("key", 0), bad.get("m", 2), bad.get("t", 32), 0, 0, 0)
        with pytest.raises(api.BMError) as e:
            api.bm_bootstrap_batch([toy.ek], j, d, d, d, ws)
        assert e.value.code == -1
    j = _uniform_jobs(api, 4, kp.n, 32, 2)
    small = api.workspace(16)
    with pytest.raises(api.BMError) as e:
        api.bm_bootstrap_batch([toy.ek], j, d, d, d, small[:16])
    assert e.value.code == -8


def test_host_buffer_entry_point_matches_device(api, orc, toy):
    kp, m, t = toy.kp, 2, 32
    cnt = 4
    _, ct = _encrypt(orc, toy, m, t, cnt, 40)
    luts, _ = synth.luts(t, cnt, 2040)
    jobs = _uniform_jobs(api, cnt, kp.n, t, m)
    dev = _run_batch(api, [toy.ek], jobs, ct, luts, cnt * (kp.n + 1))
    host_out = np.zeros(cnt * (kp.n + 1), np.uint64)
    need = api.bm_workspace_bytes([toy.ek], jobs) + api.bm_host_staging_bytes([toy.ek], jobs)
    ws = api.workspace(need + 4096)
    api.bm_bootstrap_batch_host([toy.ek], jobs, np.ascontiguousarray(ct.ravel()),
                                np.ascontiguousarray(luts.ravel()), host_out, ws)
    assert np.array_equal(host_out, dev)


def test_deterministic_repeat(api, orc, n1024):
    kp, m, t = n1024.kp, 4, 1024
    cnt = 8
    _, ct = _encrypt(orc, n1024, m, t, cnt, 50, prefix=8)
    luts, _ = synth.luts(t, cnt, 2050)
    jobs = _uniform_jobs(api, cnt, kp.n, t, m)
    a = _run_batch(api, [n1024.ek], jobs, ct, luts, cnt * (kp.n + 1))
    b = _run_batch(api, [n1024.ek], jobs, ct, luts, cnt * (kp.n + 1))
    assert np.array_equal(a, b)


# --- reusable batches: persistent launch over mixed key sets, graph replay ---------------

def _mixed_batch(api, orc, ksets, shapes, seed, prefix):
    """Jobs over several key sets; returns jobs, inputs, tables and the oracle outputs."""
    cts, luts_l, jobs, want = [], [], [], []
    in_off = lut_off = out_off = 0
    for i, (ki, m, t) in enumerate(shapes):
        ks = ksets[ki]
        kp = ks.kp
        _, ct = _encrypt(orc, ks, m, t, 1, seed + i, prefix=prefix)
        lut, _ = synth.luts(t, 1, seed + 100 + i)
        cts.append(ct[0]); luts_l.append(lut[0])
        jobs.append((ki, m, t, 0, in_off, lut_off, out_off))
        want.append(orc.bootstrap(kp, m, t, ks.bsk, ks.ksk, ct, lut)[0])
        in_off += kp.n + 1; lut_off += t; out_off += kp.n + 1
    return (np.array(jobs, dtype=api.JOB_DTYPE), np.concatenate(cts), np.concatenate(luts_l),
            want, out_off)


def test_batch_persistent_mixed_key_sets_bit_exact(api, orc, n1024, n2048):
    """Six parameter sets over the two key sets in one persistent launch."""
    shapes = [(0, 1, 256), (1, 8, 8192), (0, 2, 512), (1, 2, 2048), (0, 4, 1024), (1, 4, 4096),
              (0, 4, 1024), (1, 2, 2048), (0, 1, 256)]
    jobs, ct, luts, want, out_words = _mixed_batch(api, orc, [n1024, n2048], shapes, 60, prefix=4)
    keys = [n1024.ek, n2048.ek]
    d_in, d_lut = api.to_device_u64(ct), api.to_device_u32(luts)
    d_out = torch.zeros(out_words, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes(keys, jobs))
    b = api.Batch(keys, jobs, d_in, d_lut, d_out, ws, api.BATCH_PERSISTENT)
    b.run()
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    got = api.from_device_u64(d_out)
    for j, w in zip(jobs, want):
        o = int(j["out_off"])
        assert np.array_equal(got[o:o + len(w)], w), j
    b.free()


@pytest.mark.parametrize("flags", ["graph", "persistent+graph"])
def test_batch_graph_replay_matches_direct_path(api, orc, n1024, flags):
    kp, m, t = n1024.kp, 4, 1024
    cnt = 6
    _, ct = _encrypt(orc, n1024, m, t, cnt, 70)
    luts, _ = synth.luts(t, cnt, 2070)
    jobs = _uniform_jobs(api, cnt, kp.n, t, m)
    ref = _run_batch(api, [n1024.ek], jobs, ct, luts, cnt * (kp.n + 1))
    d_in, d_lut = api.to_device_u64(ct.ravel()), api.to_device_u32(luts.ravel())
    d_out = torch.zeros(cnt * (kp.n + 1), dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([n1024.ek], jobs))
    fl = api.BATCH_GRAPH | (api.BATCH_PERSISTENT if "persistent" in flags else 0)
    s = torch.cuda.Stream()
    b = api.Batch([n1024.ek], jobs, d_in, d_lut, d_out, ws, fl)
    for _ in range(2):
        d_out.zero_()
        torch.cuda.synchronize()
        b.run(s)
        s.synchronize()
        assert np.array_equal(api.from_device_u64(d_out), ref)
    assert api.bm_workspace_status(ws) == 0
    b.free()


def test_cluster_row_split_equals_one_block(api, orc, n1024, n2048):
    """A small batch spreads each job's rows over a thread-block cluster (up to
    8 blocks, ragged row counts, blocks with no row); one block per job
    (BATCH_ONE_BLOCK) and the oracle give the same bits."""
    shapes = [(1, 8, 8192), (0, 3, 768), (1, 2, 2048), (0, 5, 1280), (0, 1, 256), (1, 6, 6144),
              (0, 4, 1024)]
    jobs, ct, luts, want, out_words = _mixed_batch(api, orc, [n1024, n2048], shapes, 80, prefix=3)
    keys = [n1024.ek, n2048.ek]
    d_in, d_lut = api.to_device_u64(ct), api.to_device_u32(luts)
    split = api.from_device_u64(_device_run(api, keys, jobs, d_in, d_lut, out_words, None))
    one = api.from_device_u64(_device_run(api, keys, jobs, d_in, d_lut, out_words, api.BATCH_ONE_BLOCK))
    assert np.array_equal(split, one)
    for j, w in zip(jobs, want):
        o = int(j["out_off"])
        assert np.array_equal(split[o:o + len(w)], w), j


def _device_run(api, keys, jobs, d_in, d_lut, out_words, flags):
    d_out = torch.zeros(out_words, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes(keys, jobs))
    if flags is None:
        api.bm_bootstrap_batch(keys, jobs, d_in, d_lut, d_out, ws)
    else:
        b = api.Batch(keys, jobs, d_in, d_lut, d_out, ws, flags)
        b.run()
        torch.cuda.synchronize()
        b.free()
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    return d_out


# --- modulus switches and the full Algorithm 1 ----------------------------------------

def test_mod_switch_matches_oracle(api, orc, toy):
    rng = np.random.default_rng(31)
    for q_from, q_to in [(1 << 14, 1024), (toy.kp.Q, 1 << 14), (18014359854776321, 8192), (1000003, 999983)]:
        x = rng.integers(0, q_from, 4099, dtype=np.uint64)
        x[:4] = [0, q_from - 1, q_from // 2, (q_from + 1) // 2]
        d_in = api.to_device_u64(x)
        d_out = torch.zeros_like(d_in)
        api.bm_mod_switch(d_in, d_out, q_from, q_to)
        torch.cuda.synchronize()
        assert np.array_equal(api.from_device_u64(d_out), orc.mod_switch(x, q_from, q_to))


def test_full_algorithm1_with_both_modulus_switches(api, orc, toy):
    """Algorithm 1 end to end on the toy keys with q = 2^14, t = 8: switch
    q -> 2Nm = 1024, bootstrap, switch Q -> q; every message decrypts to f(msg)
    at the input modulus, and the device output equals the oracle's bits."""
    kp, m, t, q = toy.kp, 2, 8, 1 << 14
    qp = 2 * kp.N * m
    msg = np.arange(t, dtype=np.uint32)
    enc = synth.encryption_randomness(kp.n, q, kp.sigma, t, 4040)
    ct = orc.encrypt(kp.n, q, t, toy.rnd["s"], msg, enc["mask"], enc["err"])
    luts, _ = synth.luts(t, t, 2040)
    jobs = _uniform_jobs(api, t, kp.n, t, m)
    d_ct = api.to_device_u64(ct.ravel())
    d_sw = torch.zeros_like(d_ct)
    api.bm_mod_switch(d_ct, d_sw, q, qp)
    d_out = torch.zeros(t * (kp.n + 1), dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([toy.ek], jobs))
    api.bm_bootstrap_batch([toy.ek], jobs, d_sw, api.to_device_u32(luts.ravel()), d_out, ws)
    d_fin = torch.zeros_like(d_out)
    api.bm_mod_switch(d_out, d_fin, kp.Q, q)
    torch.cuda.synchronize()
    got = api.from_device_u64(d_fin).reshape(t, kp.n + 1)
    sw = orc.mod_switch(ct, q, qp)
    want = orc.mod_switch(orc.bootstrap(kp, m, t, toy.bsk, toy.ksk, sw, luts), kp.Q, q)
    assert np.array_equal(got, want)
    assert np.array_equal(api.bm_decrypt(toy.sk, q, t, got), luts[np.arange(t), msg])


def test_two_round_arbitrary_function_matches_oracle(api, orc, toy):
    """Non-negacyclic f by two rounds (one table per ciphertext), inputs with
    either top bit: bit-exact with the oracle, decrypting to f(x mod t)."""
    kp, m, t, q = toy.kp, 2, 4, 1 << 14
    T = 2 * t
    cnt = 2 * T
    x = np.tile(np.arange(T, dtype=np.uint32), 2)
    rng = np.random.default_rng(91)
    f = rng.integers(0, t, (cnt, t)).astype(np.uint32)
    f[0] = np.arange(t)                                 # identity
    enc = synth.encryption_randomness(kp.n, q, kp.sigma, cnt, 4091)
    ct = orc.encrypt(kp.n, q, T, toy.rnd["s"], x, enc["mask"], enc["err"])
    d_in = api.to_device_u64(ct.ravel())
    d_out = torch.zeros_like(d_in)
    ws = api.workspace(api.bm_arbitrary_workspace_bytes(toy.ek, m, t, cnt))
    api.bm_bootstrap_arbitrary(toy.ek, m, t, q, api.to_device_u32(f.ravel()), cnt, d_in, d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    got = api.from_device_u64(d_out).reshape(cnt, kp.n + 1)
    assert np.array_equal(got, orc.bootstrap_arbitrary(kp, m, t, q, toy.bsk, toy.ksk, ct, f))
    assert np.array_equal(api.bm_decrypt(toy.sk, q, T, got), f[np.arange(cnt), x % t])


def test_sweep_key_shape_bit_exact(api, orc):
    """The plaintext-size sweep's key shape (N = 2048, log Q = 54, B = 2^15 x 4
    digits, key-switching base 2^5 x 8), with n = 16 so the oracle stays fast:
    bootstraps and the two-round identity are bit-exact with the oracle."""
    kq = P.KEYS_SWEEP_N2048
    kp = P.KeyParams(n=16, N=kq.N, Q=kq.Q, log2_B=kq.log2_B, l_B=kq.l_B, log2_Bks=kq.log2_Bks,
                     l_ks=kq.l_ks)
    ks = KeySet(api, orc, kp, 1006, kp.n)
    shapes = [(0, 2, 64), (0, 4, 256)]
    jobs, ct, luts, want, out_words = _mixed_batch(api, orc, [ks], shapes, 90, prefix=None)
    got = api.from_device_u64(_device_run(api, [ks.ek], jobs, api.to_device_u64(ct), api.to_device_u32(luts),
                                          out_words, None))
    for j, w in zip(jobs, want):
        o = int(j["out_off"])
        assert np.array_equal(got[o:o + len(w)], w), j
    m, t = 2, 32
    q = 2 * kp.N * m
    x = np.array([3, 40], dtype=np.uint32)
    f = np.tile(np.arange(t, dtype=np.uint32), (2, 1))
    enc = synth.encryption_randomness(kp.n, q, kp.sigma, 2, 4092)
    cti = orc.encrypt(kp.n, q, 2 * t, ks.rnd["s"], x, enc["mask"], enc["err"])
    d_in = api.to_device_u64(cti.ravel())
    d_out = torch.zeros_like(d_in)
    ws = api.workspace(api.bm_arbitrary_workspace_bytes(ks.ek, m, t, 2))
    api.bm_bootstrap_arbitrary(ks.ek, m, t, q, api.to_device_u32(f.ravel()), 2, d_in, d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    out = api.from_device_u64(d_out).reshape(2, kp.n + 1)
    assert np.array_equal(out, orc.bootstrap_arbitrary(kp, m, t, q, ks.bsk, ks.ksk, cti, f))
    assert np.array_equal(api.bm_decrypt(ks.sk, q, 2 * t, out), x % t)


def test_empty_batches_are_no_ops(api, toy):
    """Zero jobs: the batch call and the two-round call return success and
    write nothing; a reusable batch of zero jobs is refused."""
    jobs = np.zeros(0, dtype=api.JOB_DTYPE)
    d_in = api.to_device_u64(np.arange(65, dtype=np.uint64))
    d_lut = api.to_device_u32(np.zeros(32, np.uint32))
    d_out = torch.full((65,), 7, dtype=torch.int64, device="cuda")
    ws = api.workspace(api.bm_workspace_bytes([toy.ek], jobs))
    api.bm_bootstrap_batch([toy.ek], jobs, d_in, d_lut, d_out, ws)
    api.bm_bootstrap_arbitrary(toy.ek, 2, 4, 1 << 14, d_lut, 0, d_in, d_out, ws)
    torch.cuda.synchronize()
    assert api.bm_workspace_status(ws) == 0
    assert bool((d_out == 7).all())
    with pytest.raises(api.BMError):
        api.Batch([toy.ek], jobs, d_in, d_lut, d_out, ws)


def test_blind_rotate_plaintext_space_fills_the_exponents(api, orc, toy):
    """t = 2Nm, the largest plaintext the test vector holds (one table entry
    per exponent of the orbit, Delta = 1): still bit-exact."""
    kp, m = toy.kp, 2
    t = 2 * kp.N * m
    _, ct = _encrypt(orc, toy, m, t, 2, 77, prefix=3)
    luts, _ = synth.luts(t, 2, 2077)
    jobs = _uniform_jobs(api, 2, kp.n, t, m)
    got = _blind_rotate_gpu(api, toy, jobs, ct, luts, 1 << 30)
    for i in range(2):
        assert np.array_equal(got[i], orc.blind_rotate(kp, m, t, toy.bsk, ct[i], luts[i])), i


def test_prefix_parity_1024_ciphertexts(api, orc, n1024):
    """1024 ciphertexts of the n = 630, N = 1024, m = 4 set whose masks vanish
    after 8 entries: ACC after the 8 CMux steps equals the oracle's on sampled
    jobs; the full bootstraps of all 1024 agree between the grouped and the
    persistent launch and decrypt to f(Dec(input))."""
    kp, m, t, cnt = n1024.kp, 4, 1024, 1024
    _, ct = _encrypt(orc, n1024, m, t, cnt, 88, prefix=8)
    luts, _ = synth.luts(t, cnt, 2088)
    jobs = _uniform_jobs(api, cnt, kp.n, t, m)
    acc = _blind_rotate_gpu(api, n1024, jobs, ct, luts, 8)
    for i in (0, 511, 1023):
        assert np.array_equal(acc[i], orc.blind_rotate(kp, m, t, n1024.bsk, ct[i], luts[i])), i
    W = kp.n + 1
    grouped = _run_batch(api, [n1024.ek], jobs, ct, luts, cnt * W)
    d_in, d_lut = api.to_device_u64(ct.ravel()), api.to_device_u32(luts.ravel())
    persistent = api.from_device_u64(_device_run(api, [n1024.ek], jobs, d_in, d_lut, cnt * W,
                                                 api.BATCH_PERSISTENT))
    assert np.array_equal(grouped, persistent)
    dec_in = api.bm_decrypt(n1024.sk, 2 * kp.N * m, t, ct)
    dec_out = api.bm_decrypt(n1024.sk, kp.Q, t, grouped.reshape(cnt, W))
    assert np.array_equal(dec_out, luts[np.arange(cnt), dec_in])
