"""Writes the full-length expected outputs of tests/test_gpu_full_length.py.

Every value stored here comes from the oracle (oracle/): Algorithm 1 with all
n CMux steps (every mask entry of every input nonzero in general), sample
extraction and key switching, computed by oracle.bootstrap on keys and
ciphertexts drawn from seeds by the oracle's own Philox4x32-10 streams
(oracle.seeded_key_randomness, oracle.encrypt_seeded).  Messages and look-up
tables come from the seeded input generator (paper_2310_12441_gb300.synth),
which draws numbers and does none of the method's arithmetic; their SHA-256
is stored so a platform whose generator stream differed would be detected.

Cases (one JSON file each):
  n630_N1024_m4    two ciphertexts, t = 2^10, random tables
  n630_N4096_m1    the same two ciphertexts (same seed, same s, q' = 8192) in
                   the single-polynomial layout
  n750_N2048_m8    two ciphertexts, t = 2^13, one random and one identity table
  uneven_S1..S6    one ciphertext per parameter set of the uneven batch

Usage: python tests/golden/make_full_length.py [case ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2310_12441_gb300 import params as P  # noqa: E402
from paper_2310_12441_gb300 import synth  # noqa: E402

CITATION = ("Algorithm 1 of arXiv 2310.12441 (ACC <- P(b)(0, v_test floor(Q/t)), all n CMux "
            "steps of Eq. (cmux:BP), sample extraction Eq. (equ-sam-extr), key switching "
            "Eq. (equ-key-swi)), computed by the CPU oracle")

KEY_SEEDS = {"n630_N1024": 1002, "n630_N4096": 1002, "n750_N2048": 1003}
KEYS = {"n630_N1024": P.KEYS_N1024, "n630_N4096": P.KEYS_N4096, "n750_N2048": P.KEYS_N2048}


def _case_specs():
    specs = {
        "n630_N1024_m4": dict(key="n630_N1024", m=4, t=1024, count=2, msg_seed=3900, enc_seed=4900,
                              lut_seed=2900, lut_mix="random"),
        "n630_N4096_m1": dict(key="n630_N4096", m=1, t=1024, count=2, msg_seed=3900, enc_seed=4900,
                              lut_seed=2900, lut_mix="random"),
        "n750_N2048_m8": dict(key="n750_N2048", m=8, t=8192, count=2, msg_seed=3901, enc_seed=4901,
                              lut_seed=2901, lut_mix="mixed"),
    }
    for i, (name, kp, shape) in enumerate(P.UNEVEN_SETS):
        key = "n630_N1024" if kp is P.KEYS_N1024 else "n750_N2048"
        specs[f"uneven_{name}"] = dict(key=key, m=shape.m, t=shape.t, count=1, msg_seed=3910 + i,
                                       enc_seed=4910 + i, lut_seed=2910 + i, lut_mix="random")
    return specs


def inputs(spec):
    """Messages and tables of a case (the seeded input generator)."""
    t, cnt = spec["t"], spec["count"]
    luts, ident = synth.luts(t, cnt, spec["lut_seed"], mix=spec["lut_mix"])
    msg = synth.messages(t, cnt, spec["msg_seed"], half=ident)
    return msg, luts


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


_key_cache = {}


def oracle_keys(key: str):
    if key not in _key_cache:
        kp = KEYS[key]
        t0 = time.time()
        rnd = oracle.seeded_key_randomness(kp, KEY_SEEDS[key])
        bsk = oracle.keygen_bsk(kp, rnd)
        ksk = oracle.keygen_ksk(kp, rnd)
        _key_cache.clear()
        _key_cache[key] = (rnd["s"], bsk, ksk)
        print(f"  keys {key}: {time.time() - t0:.0f} s", flush=True)
    return _key_cache[key]


def make(name: str, spec: dict) -> dict:
    kp = KEYS[spec["key"]]
    m, t = spec["m"], spec["t"]
    qp = 2 * kp.N * m
    s, bsk, ksk = oracle_keys(spec["key"])
    msg, luts = inputs(spec)
    ct = oracle.encrypt_seeded(kp.n, qp, t, s, msg, kp.sigma, spec["enc_seed"])
    out = []
    t0 = time.time()
    for i in range(spec["count"]):
        out.append(oracle.bootstrap(kp, m, t, bsk, ksk, ct[i:i + 1], luts[i:i + 1])[0])
    dt = time.time() - t0
    out = np.array(out, dtype=np.uint64)
    dec_in = oracle.decrypt(kp.n, qp, t, s, ct)
    dec_out = oracle.decrypt(kp.n, kp.Q, t, s, out)
    assert np.array_equal(dec_out, luts[np.arange(len(msg)), dec_in]), name
    nonzero = int((ct[:, :kp.n] != 0).sum())
    print(f"  {name}: {spec['count']} bootstraps in {dt:.0f} s, {nonzero} nonzero mask entries", flush=True)
    return {
        "case": name, "citation": CITATION, "script": "tests/golden/make_full_length.py",
        "key_set": spec["key"], "key_seed": KEY_SEEDS[spec["key"]],
        "params": {"n": kp.n, "N": kp.N, "Q": kp.Q, "log2_B": kp.log2_B, "l_B": kp.l_B,
                   "log2_Bks": kp.log2_Bks, "l_ks": kp.l_ks, "secret": kp.secret, "sigma": kp.sigma},
        "m": m, "t": t, "q_prime": qp, "count": spec["count"],
        "msg_seed": spec["msg_seed"], "enc_seed": spec["enc_seed"], "lut_seed": spec["lut_seed"],
        "lut_mix": spec["lut_mix"],
        "messages": [int(x) for x in msg], "messages_decrypted": [int(x) for x in dec_in],
        "lut_sha256": sha(luts), "ct_sha256": sha(ct),
        "nonzero_mask_entries": nonzero, "oracle_seconds": round(dt, 1),
        "out": ["".join(f"{int(w):016x}" for w in row) for row in out],
    }


def main(argv):
    specs = _case_specs()
    names = argv or list(specs)
    # keep cases of one key set together (the oracle keys are rebuilt per key set)
    names.sort(key=lambda nm: (specs[nm]["key"], nm))
    for nm in names:
        print(f"case {nm}", flush=True)
        d = make(nm, specs[nm])
        with open(os.path.join(HERE, f"full_length_{nm}.json"), "w") as f:
            json.dump(d, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
