"""Every kernel shape the autotuner may pick (NTT radix, threads per block,
blocks per SM) gives the oracle's bits: per ring degree of the production
key sets, through grouped launches, thread-block clusters (small batches),
one block per job, and the persistent kernels where the shape allows them."""
import numpy as np
import pytest

from paper_2310_12441_gb300 import params as P
from paper_2310_12441_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(P.KEYS_N1024, 4, 1024), (P.KEYS_N2048, 8, 8192), (P.KEYS_N4096, 1, 1024)]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_12441_gb300 import api as A
    A.load()
    yield A
    for N in (1024, 2048, 4096):
        A.set_kernel_shape(N, A.SHAPE_DEFAULT)


@pytest.mark.parametrize("kp,m,t", CASES, ids=["N1024_m4", "N2048_m8", "N4096_m1"])
def test_every_shape_matches_the_oracle(api, orc, kp, m, t):
    prefix = 3
    seed = 1300 + kp.N
    sk, ek = api.bm_keygen_seeded(kp, seed)
    rnd = orc.seeded_key_randomness(kp, seed, bsk_keys=prefix)
    bsk, ksk = orc.keygen_bsk(kp, rnd), orc.keygen_ksk(kp, rnd)
    qp = 2 * kp.N * m
    cnt = 3
    msg = synth.messages(t, cnt, seed)
    ct = api.bm_encrypt_seeded(sk, qp, t, msg, seed + 1)
    ct[:, prefix:kp.n] = 0
    luts, _ = synth.luts(t, cnt, seed + 2)
    want = orc.bootstrap(kp, m, t, bsk, ksk, ct, luts)
    W = kp.n + 1
    jobs = api.make_jobs(0, m, t, np.arange(cnt) * W, np.arange(cnt) * t, np.arange(cnt) * W)
    d_in, d_lut = api.to_device_u64(ct.ravel()), api.to_device_u32(luts.ravel())
    shapes = api.kernel_shapes(kp.N)
    assert 0 in shapes and 1 in shapes
    for sh, (radix, threads, blocks) in shapes.items():
        api.set_kernel_shape(kp.N, sh)
        assert api.get_kernel_shape(kp.N) == sh
        forms = [None, api.BATCH_ONE_BLOCK] + ([api.BATCH_PERSISTENT] if blocks == 1 else [])
        for flags in forms:
            d_out = torch.zeros(cnt * W, dtype=torch.int64, device="cuda")
            ws = api.workspace(api.bm_workspace_bytes([ek], jobs))
            if flags is None:
                api.bm_bootstrap_batch([ek], jobs, d_in, d_lut, d_out, ws)     # clusters (3 jobs)
            else:
                b = api.Batch([ek], jobs, d_in, d_lut, d_out, ws, flags)
                b.run()
                torch.cuda.synchronize()
                b.free()
            torch.cuda.synchronize()
            assert api.bm_workspace_status(ws) == 0
            got = api.from_device_u64(d_out).reshape(cnt, W)
            assert np.array_equal(got, want), (sh, radix, threads, blocks, flags)
    api.set_kernel_shape(kp.N, api.SHAPE_DEFAULT)
