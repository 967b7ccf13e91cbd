"""Parity at the benchmark's full sizes, built the way bench.py builds them
(wt_build_async, automatic variant, default stream).

At 2^30 symbols the oracle cannot rebuild whole trees in seconds, so these
tests check what fixes every level at any size, against exact counts taken
from S itself:
  * level 0 is the top bit of every symbol (Proposition 1 with l = 0), and
    its rank directory is the running count of those bits;
  * the ones of level l are the symbols whose bit l is set (a histogram
    sum), for every level;
  * access(i) == S[i], rank_c(i) and select_c(j) equal direct counting on S,
    on sampled arguments; these walk every level's bitmap and rank and
    select directories (Section 2.2).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import needs_gpu, wt
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]

BLOCK = 1 << 16


class Occurrences:
    """Exact rank/select of one symbol c in S from per-block counts."""

    def __init__(self, S: np.ndarray, c: int):
        self.S, self.c = S, c
        eq = S == c
        nb = (len(S) + BLOCK - 1) // BLOCK
        pad = np.zeros(nb * BLOCK, dtype=np.uint8)
        pad[: len(S)] = eq
        per = pad.reshape(nb, BLOCK).sum(axis=1, dtype=np.int64)
        self.cum = np.concatenate([[0], np.cumsum(per)])
        self.count = int(self.cum[-1])

    def rank(self, i: int) -> int:
        b = i // BLOCK
        return int(self.cum[b] + np.count_nonzero(self.S[b * BLOCK: i] == self.c))

    def select(self, j: int) -> int:
        if j < 1 or j > self.count:
            return 2**64 - 1
        b = int(np.searchsorted(self.cum, j, side="left")) - 1
        pos = np.flatnonzero(self.S[b * BLOCK: (b + 1) * BLOCK] == self.c)
        return b * BLOCK + int(pos[j - self.cum[b] - 1])


def check_full(W, S: np.ndarray, sigma: int, seed: int):
    n = len(S)
    L = (sigma - 1).bit_length()
    dev = torch.from_numpy(S).cuda()
    tree = W.Tree.build(dev, sigma, wait=False)
    tree.wait()
    del dev
    # ones of every level from the histogram
    hist = np.bincount(S, minlength=sigma).astype(np.int64)
    codes = np.arange(sigma, dtype=np.int64)
    for l in range(L):
        want = int(hist[((codes >> (L - 1 - l)) & 1) == 1].sum())
        assert tree.level(l).ones == want, f"level {l} ones"
    # level 0 = top bits of S, and its block directory
    top = ((S >> (L - 1)) & 1).astype(np.uint8)
    lb = ((n + 511) // 512) * 64
    bits0 = np.zeros(lb * 8, dtype=np.uint8)
    bits0[:n] = top
    want0 = np.packbits(bits0, bitorder="little")
    lv0 = tree.level(0)
    assert np.array_equal(lv0.words.cpu().numpy().view(np.uint8), want0)
    per_block = bits0.reshape(-1, 512).sum(axis=1, dtype=np.int64)
    R = np.concatenate([[0], np.cumsum(per_block)]) % (1 << 32)
    assert np.array_equal(lv0.R.cpu().numpy().astype(np.int64), R)
    # queries against exact counts on S
    rng = np.random.default_rng(seed)
    m = 4096
    I = rng.integers(0, n, m).astype(np.uint64)
    I[:2] = [0, n - 1]
    got = tree.access(torch.from_numpy(I).cuda()).cpu().numpy()
    assert np.array_equal(got.astype(np.int64), S[I.astype(np.int64)].astype(np.int64))
    present = np.flatnonzero(hist)
    picks = {int(np.argmax(hist)), int(present[np.argmin(hist[present])]), int(present[len(present) // 2])}
    for c in sorted(picks):
        occ = Occurrences(S, c)
        ii = np.concatenate([[0, n], rng.integers(0, n + 1, 64)]).astype(np.uint64)
        jj = np.concatenate([[1, occ.count, occ.count + 1], rng.integers(1, occ.count + 1, 64)]).astype(np.uint64)
        cc = np.full(len(ii), c, np.uint32)
        r = tree.rank(torch.from_numpy(cc).cuda(), torch.from_numpy(ii).cuda()).cpu().numpy()
        assert [int(v) for v in r] == [occ.rank(int(i)) for i in ii], f"rank of {c}"
        cj = np.full(len(jj), c, np.uint32)
        s = tree.select(torch.from_numpy(cj).cuda(), torch.from_numpy(jj).cuda()).cpu().numpy()
        assert [int(v) for v in s] == [occ.select(int(j)) for j in jj], f"select of {c}"
    tree.free()


@pytest.mark.parametrize("name", ["u8-text-2^30-s96-zipf1.0", "u8-dna-2^30-s4", "u32-words-2^29-s2^20-zipf1.2"])
def test_full_size_workload(name):
    W = wt()
    w = inputs.WORKLOADS[name]
    S = w.generate()
    check_full(W, S, w.sigma, seed=len(name))
    torch.cuda.empty_cache()
