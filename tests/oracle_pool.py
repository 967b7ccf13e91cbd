"""The CPU oracle on several host cores, for parity checks at full size.

Test helper (imports no torch): the workers run the oracle of ``oracle/``
and nothing else.  Pools are started with the spawn method, because the test
process already holds a CUDA context and a forked child of it can hang.

* ``tree_levels`` gives, level by level, the bitmap of one long sequence by
  Algorithm 1's per-level body (levels are independent there) and its
  directory, for the long single-sequence workloads (2^29 .. 2^30 symbols).
* ``batch_digests`` gives, for many generated sequences, a digest of every
  level's bitmap, directory and ones count, computed from the oracle's whole
  tree of each sequence; the test computes the same digest from the GPU tree.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
import tempfile

import numpy as np

from oracle import oracle as O


def _mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def _workers(tasks: int, bytes_per_worker: int) -> int:
    cores = os.cpu_count() or 1
    mem = max(1, int(_mem_available() * 0.6) // max(1, bytes_per_worker))
    return max(1, min(tasks, cores, mem))


def _one_level(args):
    path, sigma, l = args
    S = np.load(path, mmap_mode="r")
    bits = O.pwt_level_bits(S, sigma, l)
    return l, bits, O.directory(bits, len(S))


def tree_levels(S: np.ndarray, sigma: int):
    """Yields (l, bitmap bytes, directory dict) for every level of S's tree,
    in completion order, computed in a spawn-started process pool."""
    L = O.levels(sigma)
    if L == 0:
        return
    n = len(S)
    per = n * S.itemsize + 4 * n + 2 * O.level_bytes(n)   # the mapped S, the oracle's codes, a bitmap
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "S.npy")
        np.save(path, S)
        ctx = mp.get_context("spawn")
        with ctx.Pool(_workers(L, per)) as pool:
            for res in pool.imap_unordered(_one_level, [(path, sigma, l) for l in range(L)]):
                yield res


def level_digest(words: np.ndarray, R: np.ndarray, Hy: np.ndarray, S1: np.ndarray, S0: np.ndarray, ones: int) -> str:
    """One digest of a level's bitmap bytes and directory arrays."""
    h = hashlib.blake2b(digest_size=20)
    for a, dt in ((words, np.uint8), (R, np.uint32), (Hy, np.uint64), (S1, np.uint32), (S0, np.uint32)):
        h.update(np.ascontiguousarray(a).view(dt).tobytes())
        h.update(b"|")
    h.update(int(ones).to_bytes(8, "little"))
    return h.hexdigest()


def _seq_digests(specs):
    out = []
    for sp in specs:
        S = sp.generate()
        bits = O.build_bits(S, sp.sigma)
        digests = []
        for l in range(bits.shape[0]):
            d = O.directory(bits[l], len(S))
            digests.append(level_digest(bits[l], d["R"], d["Hy"], d["S1"], d["S0"], d["ones"]))
        out.append(digests)
    return out


def batch_digests(specs, chunk: int = 32):
    """Per sequence of specs (SeqSpec), the list of its levels' digests from
    the oracle's tree, computed in a spawn-started process pool."""
    groups = [specs[i:i + chunk] for i in range(0, len(specs), chunk)]
    biggest = max((sp.n for sp in specs), default=1)
    per = biggest * 24 + (64 << 20)
    ctx = mp.get_context("spawn")
    with ctx.Pool(_workers(len(groups), per)) as pool:
        parts = pool.map(_seq_digests, groups)
    return [d for part in parts for d in part]
