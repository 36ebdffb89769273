"""Assembles bootstrapping batches from seeded synthetic inputs.

A batch is a list of jobs (bm_job records) with their input ciphertexts,
look-up tables and expected plaintexts.  Keys and encryptions come from the
library's seeded entry points; messages and tables from synth.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import api, synth
from .params import JobShape, KeyParams


@dataclass
class KeySet:
    kp: KeyParams
    sk: api.SecretKey
    ek: api.EvalKey
    seed: int


def make_keyset(kp: KeyParams, seed: int, device: int = 0) -> KeySet:
    """Keys from a seed, the evaluation key drawn and built on the device."""
    sk, ek = api.bm_keygen_seeded(kp, seed, device)
    return KeySet(kp, sk, ek, seed)


@dataclass
class Batch:
    jobs: np.ndarray          # JOB_DTYPE
    ct_in: np.ndarray         # uint64 words
    luts: np.ndarray          # uint32 words
    out_words: int
    msg: np.ndarray           # plaintext of each job
    dec_in: np.ndarray        # Dec(input) of each job (what the output must decrypt to under f)
    expect: np.ndarray        # f(Dec(input)) for each job
    key_of: np.ndarray        # key-set index of each job


def make_batch(keysets: list[KeySet], groups: list[tuple[int, JobShape, int]], seed: int,
               lut_mix: str = "random", interleave: bool = True) -> Batch:
    """groups: (key-set index, shape, count).  interleave=True shuffles the jobs
    of all groups (seeded) so no launch sees them sorted."""
    parts = []
    for g, (ki, shape, count) in enumerate(groups):
        if count == 0:
            continue
        ks = keysets[ki]
        kp = ks.kp
        m, t = shape.m, shape.t
        qp = 2 * kp.N * m
        luts, ident = synth.luts(t, count, 2000 + seed + 17 * g, mix=lut_mix)
        msg = synth.messages(t, count, 3000 + seed + 17 * g, half=ident)
        ct = api.bm_encrypt_seeded(ks.sk, qp, t, msg, 4000 + seed + 17 * g)
        dec = api.bm_decrypt(ks.sk, qp, t, ct)
        for i in range(count):
            parts.append((ki, m, t, ct[i], luts[i], msg[i], dec[i], luts[i][dec[i]]))
    order = np.arange(len(parts))
    if interleave:
        np.random.default_rng(seed).shuffle(order)
    jobs = np.zeros(len(parts), api.JOB_DTYPE)
    cts, lts = [], []
    in_off = lut_off = out_off = 0
    msg = np.zeros(len(parts), np.uint32)
    dec = np.zeros(len(parts), np.uint32)
    exp = np.zeros(len(parts), np.uint32)
    key_of = np.zeros(len(parts), np.int32)
    for j, idx in enumerate(order):
        ki, m, t, ct, lut, mm, dd, ee = parts[idx]
        n = keysets[ki].kp.n
        jobs[j] = (ki, m, t, 0, in_off, lut_off, out_off)
        cts.append(ct)
        lts.append(lut)
        msg[j], dec[j], exp[j], key_of[j] = mm, dd, ee, ki
        in_off += n + 1
        lut_off += t
        out_off += n + 1
    return Batch(jobs, np.concatenate(cts).astype(np.uint64), np.concatenate(lts).astype(np.uint32),
                 out_off, msg, dec, exp, key_of)


def check_outputs(keysets: list[KeySet], batch: Batch, out: np.ndarray) -> int:
    """Number of outputs that do not decrypt (at Q) to f(Dec(input))."""
    bad = 0
    for ki, ks in enumerate(keysets):
        sel = np.nonzero(batch.key_of == ki)[0]
        if sel.size == 0:
            continue
        n = ks.kp.n
        offs = batch.jobs["out_off"][sel].astype(np.int64)
        cts = np.stack([out[o:o + n + 1] for o in offs])
        ts = batch.jobs["t"][sel]
        for t in np.unique(ts):
            s2 = ts == t
            dec = api.bm_decrypt(ks.sk, ks.kp.Q, int(t), cts[s2])
            bad += int((dec != batch.expect[sel][s2]).sum())
    return bad
