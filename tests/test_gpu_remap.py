"""Trees over non-contiguous alphabets (wt_build_remap; Section 3's remap of
the sequence to a contiguous alphabet through a bitmap): the alphabet bitmap
and its directory, every level of the tree of the remapped sequence, and
access/rank/select on original codes equal the CPU oracle's."""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, to_dev, wt
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, needs_gpu]


def _sample(alphabet, n, seed, dtype):
    rng = np.random.default_rng(seed)
    a = np.asarray(sorted(alphabet), dtype=np.uint64)
    w = 1.0 / np.arange(1, len(a) + 1) ** 1.1          # skewed use of the codes
    idx = rng.choice(len(a), size=n, p=w / w.sum())
    return a[idx].astype(dtype)


def _queries(S, universe, codes, m, seed):
    rng = np.random.default_rng(seed)
    n = len(S)
    I = rng.integers(0, n + 2, m).astype(np.uint64)
    extra = [c for c in (0, 1, universe - 1, universe, universe + 3) if c < 2**32]
    C = np.concatenate([S[rng.integers(0, max(n, 1), m - len(extra))].astype(np.uint64) if n else
                        np.zeros(m - len(extra), np.uint64), np.asarray(extra, np.uint64)])
    counts = {int(c): int(np.sum(S == c)) for c in np.unique(C)}
    J = np.array([rng.integers(0, counts[int(c)] + 2) for c in C], dtype=np.uint64)
    return I, C.astype(np.uint32), J


@pytest.mark.parametrize("universe,ncodes,dtype,n", [
    (1 << 20, 50, np.uint32, 100_003), (65536, 300, np.uint16, 70_001), (256, 4, np.uint8, 5003),
    (1 << 24, 3000, np.uint32, (1 << 20) + 7), (256, 256, np.uint8, 9001), (5, 1, np.uint8, 100),
    (1 << 16, 70, np.uint16, 1)])
def test_remapped_tree_equals_the_oracle(universe, ncodes, dtype, n):
    W = wt()
    rng = np.random.default_rng(universe + ncodes)
    alphabet = rng.choice(universe, size=ncodes, replace=False)
    S = _sample(alphabet, n, n, dtype)
    bm, codes, Sr, sr = O.remap_alphabet(S, universe)
    t = W.Tree.build_remap(to_dev(S), universe)
    info = t.info()
    assert info["universe"] == universe and info["sigma"] == sr
    A = t.alphabet()
    assert np.array_equal(A.words.cpu().numpy().view(np.uint8), bm)
    d = O.directory(bm, universe)
    for key, arr in (("R", A.R), ("Hy", A.Hy), ("S1", A.S1), ("S0", A.S0)):
        assert np.array_equal(arr.cpu().numpy(), d[key]), key
    assert A.ones == len(codes)
    bits = compare_tree(t, Sr, sr)
    I, C, J = _queries(S, universe, codes, 3000, n)
    got = t.access(to_dev(I)).cpu().numpy()
    assert np.array_equal(got, O.remap_access(codes, bits, n, sr, I))
    got = t.rank(to_dev(C), to_dev(I)).cpu().numpy()
    assert np.array_equal(got, O.remap_rank(codes, universe, bits, n, sr, C, I))
    got = t.select(to_dev(C), to_dev(J)).cpu().numpy()
    assert np.array_equal(got, O.remap_select(codes, universe, bits, n, sr, C, J))
    t.free()


def test_remap_over_the_whole_32_bit_universe():
    """Sparse 32-bit ids (the bitmap covers 2^32 codes): levels equal the
    oracle's tree of the dense ranks, queries equal direct counting on S."""
    W = wt()
    alphabet = [0, 7, 1000, 1 << 31, (1 << 32) - 1]
    S = _sample(alphabet, 10_007, 5, np.uint32)
    t = W.Tree.build_remap(to_dev(S), 1 << 32)
    codes = np.unique(S).astype(np.uint64)
    Sr = np.searchsorted(codes, S.astype(np.uint64)).astype(np.uint32)
    assert t.info()["sigma"] == len(codes)
    compare_tree(t, Sr, len(codes))
    n = len(S)
    I = np.arange(0, n + 2, 97, dtype=np.uint64)
    got = t.access(to_dev(I)).cpu().numpy()
    assert [int(x) for x in got] == [int(S[i]) if i < n else 0xFFFFFFFF for i in I]
    for c in alphabet + [5, (1 << 32) - 2]:
        Cs = np.full(len(I), c, np.uint32)
        r = t.rank(to_dev(Cs), to_dev(I)).cpu().numpy()
        assert [int(x) for x in r] == [int(np.sum(S[:i] == c)) if i <= n else 2**64 - 1 for i in I]
        occ = np.flatnonzero(S == c)
        Jv = np.array([0, 1, len(occ), len(occ) + 1], np.uint64)
        s = t.select(to_dev(np.full(4, c, np.uint32)), to_dev(Jv)).cpu().numpy()
        want = [2**64 - 1] + ([int(occ[0]), int(occ[-1])] if len(occ) else [2**64 - 1, 2**64 - 1]) + [2**64 - 1]
        assert [int(x) for x in s] == want, c
    t.free()


def test_remap_errors():
    W = wt()
    S = np.array([3, 9, 10, 3], np.uint8)
    with pytest.raises(W.WTError) as e:
        W.Tree.build_remap(to_dev(S), 10)
    assert e.value.status == W.ERR_SYMBOL_RANGE
    with pytest.raises(W.WTError) as e:
        W.Tree.build_remap(to_dev(S), 300)                    # universe beyond 1-byte codes
    assert e.value.status == W.ERR_ARG
    t = W.Tree.build_remap(to_dev(np.array([3, 9, 3], np.uint8)), 16)
    other = W.Tree.build(to_dev(np.array([1, 0, 1], np.uint8)), 2)
    q = [to_dev(np.zeros(1, np.uint32)), to_dev(np.zeros(1, np.uint8)), to_dev(np.zeros(1, np.uint32)),
         to_dev(np.zeros(1, np.uint64))]
    with pytest.raises(W.WTError) as e:
        W.query_multi([other, t], *q)
    assert e.value.status == W.ERR_ARG
    host = W.Tree.build_remap(np.array([5, 200, 5, 7], np.uint8), 256)   # host input
    assert host.info()["sigma"] == 3
    torch.cuda.synchronize()
