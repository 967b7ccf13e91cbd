"""GPU parity of queries (kernel e): access, rank and select through the C ABI
equal the oracle's answers on random and edge batches, sentinels included."""
import numpy as np
import pytest
import torch

from gpu_helpers import needs_gpu, query_batches, to_dev, wt
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def run_queries(W, tree, S, sigma, m=4096, seed=0):
    n = len(S)
    I, Cs, J = query_batches(S, sigma, m, seed)
    bits = O.build_bits(S, sigma)
    acc = tree.access(torch.from_numpy(I).cuda()).cpu().numpy()
    rk = tree.rank(torch.from_numpy(Cs).cuda(), torch.from_numpy(I).cuda()).cpu().numpy()
    sl = tree.select(torch.from_numpy(Cs).cuda(), torch.from_numpy(J).cuda()).cpu().numpy()
    assert np.array_equal(acc, O.access(bits, n, sigma, I))
    assert np.array_equal(rk, O.rank(bits, n, sigma, Cs, I))
    assert np.array_equal(sl, O.select(bits, n, sigma, Cs, J))
    return acc, rk, sl


@pytest.mark.parametrize("sigma,dtype,n", [(1, np.uint8, 1000), (2, np.uint8, 4097), (3, np.uint8, 513),
                                           (4, np.uint8, 70001), (96, np.uint8, 100_003), (256, np.uint8, 1 << 16),
                                           (20, np.uint8, 0), (65536, np.uint16, 50_000),
                                           (1 << 20, np.uint32, 30_011)])
def test_queries_match_oracle(sigma, dtype, n):
    W = wt()
    S = inputs.zipf(n, sigma, 1.0, 31 + n, dtype) if n else np.zeros(0, dtype)
    t = W.Tree.build(to_dev(S), sigma)
    run_queries(W, t, S, sigma, m=2048, seed=n)


def test_queries_brute_force_small_workload():
    """access = S[i], rank by counting, select by scanning, on the 2^20 x 256 workload."""
    W = wt()
    wl = inputs.WORKLOADS["u8-uniform-2^20-s256"]
    S = wl.generate()
    t = W.Tree.build(to_dev(S), wl.sigma)
    rng = np.random.default_rng(5)
    I = rng.integers(0, len(S), 3000).astype(np.uint64)
    assert np.array_equal(t.access(torch.from_numpy(I).cuda()).cpu().numpy(), S[I.astype(np.int64)])
    Cs = S[rng.integers(0, len(S), 3000)].astype(np.uint32)
    rk = t.rank(torch.from_numpy(Cs).cuda(), torch.from_numpy(I).cuda()).cpu().numpy()
    pos = {c: np.flatnonzero(S == c) for c in np.unique(Cs)}
    want = np.array([np.searchsorted(pos[c], i) for c, i in zip(Cs, I)], dtype=np.uint64)
    assert np.array_equal(rk, want)
    J = np.array([rng.integers(1, len(pos[c]) + 1) for c in Cs], dtype=np.uint64)
    sl = t.select(torch.from_numpy(Cs).cuda(), torch.from_numpy(J).cuda()).cpu().numpy()
    assert np.array_equal(sl, np.array([pos[c][j - 1] for c, j in zip(Cs, J)], dtype=np.uint64))


def test_select_inverts_rank_on_device():
    W = wt()
    sigma = 96
    S = inputs.zipf(300_001, sigma, 1.0, 3, np.uint8)
    t = W.Tree.build(to_dev(S), sigma)
    I = np.arange(0, len(S), 13, dtype=np.uint64)
    c = torch.from_numpy(S[I.astype(np.int64)].astype(np.uint32)).cuda()
    r = t.rank(c, torch.from_numpy(I).cuda())
    back = t.select(c, torch.from_numpy(r.cpu().numpy() + np.uint64(1)).cuda()).cpu().numpy()
    assert np.array_equal(back, I)


def test_query_multi_over_several_trees():
    W = wt()
    rng = np.random.default_rng(9)
    specs = [(256, np.uint8, 40_000), (65536, np.uint16, 30_000), (4, np.uint8, 50_001)]
    trees, seqs = [], []
    for k, (sigma, dt, n) in enumerate(specs):
        S = inputs.zipf(n, sigma, 1.0, 100 + k, dt)
        seqs.append(S)
        trees.append(W.Tree.build(to_dev(S), sigma))
    m = 6000
    tidx = rng.integers(0, len(trees), m).astype(np.uint32)
    op = rng.integers(0, 3, m).astype(np.uint8)
    c = np.zeros(m, np.uint32)
    arg = np.zeros(m, np.uint64)
    want = np.zeros(m, np.uint64)
    for q in range(m):
        S = seqs[tidx[q]]
        sigma = specs[tidx[q]][0]
        c[q] = S[rng.integers(0, len(S))]
        if op[q] == 2:
            arg[q] = rng.integers(0, int(np.sum(S == c[q])) + 2)
        else:
            arg[q] = rng.integers(0, len(S) + 2)
    for k, (S, (sigma, _, n)) in enumerate(zip(seqs, specs)):
        sel = tidx == k
        bits = O.build_bits(S, sigma)
        a = O.access(bits, n, sigma, arg[sel & (op == 0)]).astype(np.uint64)
        a[a == 0xFFFFFFFF] = np.uint64(2**64 - 1)
        want[sel & (op == 0)] = a
        want[sel & (op == 1)] = O.rank(bits, n, sigma, c[sel & (op == 1)], arg[sel & (op == 1)])
        want[sel & (op == 2)] = O.select(bits, n, sigma, c[sel & (op == 2)], arg[sel & (op == 2)])
    got = W.query_multi(trees, torch.from_numpy(tidx).cuda(), torch.from_numpy(op).cuda(),
                        torch.from_numpy(c).cuda(), torch.from_numpy(arg).cuda()).cpu().numpy()
    assert np.array_equal(got, want)


def test_query_multi_tree_index_outside_the_table_gives_the_sentinel():
    """A tree index >= ntrees reads nothing and answers UINT64_MAX; the other
    queries of the batch are unaffected."""
    W = wt()
    S = inputs.zipf(20_000, 96, 1.0, 7, np.uint8)
    t = W.Tree.build(to_dev(S), 96)
    tidx = to_dev(np.array([0, 1, 7, 0xFFFFFFFF, 0], np.uint32))
    op = to_dev(np.array([0, 0, 1, 2, 1], np.uint8))
    c = to_dev(np.array([0, 0, S[5], S[5], S[5]], np.uint32))
    arg = to_dev(np.array([5, 5, 100, 1, 100], np.uint64))
    got = W.query_multi([t], tidx, op, c, arg).cpu().numpy()
    ones = np.uint64(2**64 - 1)
    assert got[1] == ones and got[2] == ones and got[3] == ones
    assert int(got[0]) == int(S[5])
    assert int(got[4]) == int(np.sum(S[:100] == S[5]))
