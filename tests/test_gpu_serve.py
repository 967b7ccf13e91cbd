"""The serving loop (continuous batching): builds admitted under a memory
budget with eviction, query batches overlapping the builds on another
stream, and every result equal to what the same request gets alone."""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, to_dev, wt
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_serving_results_equal_alone():
    W = wt()
    from paper_1610_05994_gb300.serve import BuildRequest, Server
    rng = np.random.default_rng(11)
    specs = inputs.serving_specs(40, log2_min=10, log2_max=17)
    seqs = [sp.generate() for sp in specs]
    # 3.5 MB: above the largest build's need (2.9 MB with its scratch), below
    # that plus the trees left resident (2.8 MB in all), so admission evicts.
    srv = Server(budget_bytes=7 << 19, max_batch=8)
    issued = []  # (query batch, [rid per tree], tidx, op, c, arg)
    nxt = 0
    for round_ in range(60):
        for _ in range(rng.integers(0, 3)):
            if nxt < len(specs):
                sp = specs[nxt]
                srv.submit(BuildRequest(nxt, to_dev(seqs[nxt]), sp.sigma, 0.0))
                nxt += 1
        srv.step()
        res = list(srv.resident.items())
        if res and round_ % 2 == 0:
            trees = [v[0] for _, v in res]
            rids = [rid for rid, _ in res]
            m = 1024
            tidx = rng.integers(0, len(trees), m).astype(np.uint32)
            op = rng.integers(0, 3, m).astype(np.uint8)
            c = np.zeros(m, np.uint32)
            arg = np.zeros(m, np.uint64)
            for q in range(m):
                S = seqs[rids[tidx[q]]]
                c[q] = S[rng.integers(0, len(S))]
                arg[q] = rng.integers(0, len(S) + 2) if op[q] != 2 else rng.integers(0, 40)
            qb = srv.query(trees, *(torch.from_numpy(x).cuda() for x in (tidx, op, c, arg)))
            issued.append((qb, rids, tidx, op, c, arg))
    while nxt < len(specs):
        srv.submit(BuildRequest(nxt, to_dev(seqs[nxt]), specs[nxt].sigma, 0.0))
        nxt += 1
    srv.drain()
    assert srv.evicted > 0, "the budget should have forced evictions"
    assert len(srv.finished) == len(specs)
    # query answers in the mix equal the oracle's answers for each request alone
    bits = {}
    for qb, rids, tidx, op, c, arg in issued:
        got = qb.out.cpu().numpy()
        for q in range(len(arg)):
            rid = rids[tidx[q]]
            S, sigma = seqs[rid], specs[rid].sigma
            if rid not in bits:
                bits[rid] = O.build_bits(S, sigma)
            b = bits[rid]
            if op[q] == 0:
                a = O.access(b, len(S), sigma, arg[q:q + 1])[0]
                want = 2**64 - 1 if a == 0xFFFFFFFF else int(a)
            elif op[q] == 1:
                want = int(O.rank(b, len(S), sigma, c[q:q + 1], arg[q:q + 1])[0])
            else:
                want = int(O.select(b, len(S), sigma, c[q:q + 1], arg[q:q + 1])[0])
            assert int(got[q]) == want, (rid, int(op[q]))
    # trees still resident equal the oracle's (and so a build alone)
    for rid, (tree, _, req) in list(srv.resident.items()):
        compare_tree(tree, seqs[rid], specs[rid].sigma, check_dir=False)
    srv.close()


def test_failed_and_oversized_requests_do_not_stall_the_loop():
    """A request larger than the whole budget is refused without evicting
    anything; a build that fails (a symbol >= sigma) is recorded, its bytes
    are given back, and the other builds of its batch still become resident
    with trees equal to the oracle's."""
    W = wt()
    from paper_1610_05994_gb300.serve import BuildRequest, Server, tree_bytes
    good = [inputs.zipf(5000 + 17 * k, 256, 1.0, 50 + k, np.uint8) for k in range(3)]
    bad = inputs.uniform(6000, 200, 60, np.uint8)
    bad[4321] = 250
    huge = np.zeros(1 << 20, np.uint8)
    budget = 6 * tree_bytes(len(bad) + 1000, 256, 1)   # room for all four small builds
    assert tree_bytes(len(huge), 256, 1) > budget
    srv = Server(budget_bytes=budget, max_batch=8)
    srv.submit(BuildRequest(0, to_dev(good[0]), 256, 0.0))
    srv.step()
    srv.drain()
    assert list(srv.resident) == [0]
    srv.submit(BuildRequest(1, to_dev(huge), 256, 0.0))
    srv.submit(BuildRequest(2, to_dev(good[1]), 256, 0.0))
    srv.submit(BuildRequest(3, to_dev(bad), 200, 0.0))
    srv.submit(BuildRequest(4, to_dev(good[2]), 256, 0.0))
    srv.drain()
    assert [r.rid for r in srv.rejected] == [1] and srv.rejected[0].error
    assert [r.rid for r in srv.failed] == [3] and srv.failed[0].error
    assert sorted(srv.resident) == [0, 2, 4]
    assert srv.evicted == 0
    assert srv.used == sum(v[1] for v in srv.resident.values())
    for rid, S in ((0, good[0]), (2, good[1]), (4, good[2])):
        compare_tree(srv.resident[rid][0], S, 256)
    srv.close()
