"""GPU parity of the batched build (wt_build_batch): every sequence of a
mixed batch gives exactly the oracle's tree, and exactly the tree it gets
when built alone."""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, query_batches, to_dev, tree_bits, wt
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def mixed_specs(seed=0):
    rng = np.random.default_rng(seed)
    specs = []
    shapes = [(1, np.uint8), (2, np.uint8), (4, np.uint8), (20, np.uint8), (96, np.uint8), (256, np.uint8),
              (300, np.uint16), (65536, np.uint16), (4, np.uint16), (1 << 20, np.uint32), (17, np.uint32)]
    sizes = [0, 1, 31, 513, 4097, 16385, 70001, 250_003]
    for i in range(44):
        sigma, dt = shapes[i % len(shapes)]
        n = sizes[rng.integers(0, len(sizes))]
        specs.append((sigma, dt, n))
    return specs


def make_seqs(specs, seed=1):
    seqs = []
    for k, (sigma, dt, n) in enumerate(specs):
        S = inputs.zipf(n, sigma, 1.1, seed * 1000 + k, dt) if n else np.zeros(0, dt)
        seqs.append(S)
    return seqs


@pytest.mark.parametrize("on_stream", [False, True])
def test_mixed_batch_matches_oracle_and_single_builds(on_stream):
    W = wt()
    specs = mixed_specs()
    seqs = make_seqs(specs)
    dev = [to_dev(S) for S in seqs]
    stream = torch.cuda.Stream() if on_stream else None
    torch.cuda.synchronize()
    trees = W.build_batch(dev, [s[0] for s in specs], stream=stream)
    for (sigma, _, n), S, t in zip(specs, seqs, trees):
        compare_tree(t, S, sigma)
        alone = W.Tree.build(to_dev(S), sigma, variant=W.VARIANT_LEVELWISE)
        assert np.array_equal(tree_bits(t), tree_bits(alone))
    for t in trees[::2]:
        t.free()
    # the rest still answer queries after half of the batch is gone
    for (sigma, _, n), S, t in list(zip(specs, seqs, trees))[1::2]:
        if n == 0:
            continue
        I, Cs, J = query_batches(S, sigma, 256, n)
        bits = O.build_bits(S, sigma)
        got = t.rank(torch.from_numpy(Cs).cuda(), torch.from_numpy(I).cuda()).cpu().numpy()
        assert np.array_equal(got, O.rank(bits, n, sigma, Cs, I))


def test_batch_reports_a_bad_sequence_and_builds_the_others():
    W = wt()
    good = inputs.uniform(100_000, 20, 3, np.uint8)
    bad = np.array([0, 1, 2, 25, 3], dtype=np.uint8)
    trees = W.build_batch([to_dev(good), to_dev(bad), to_dev(good)], [20, 20, 20], wait=False)
    statuses = []
    for t in trees:
        try:
            t.wait()
            statuses.append(W.OK)
        except W.WTError as e:
            statuses.append(e.status)
    assert statuses == [W.OK, W.ERR_SYMBOL_RANGE, W.OK]
    compare_tree(trees[0], good, 20)
    compare_tree(trees[2], good, 20)


def test_batch_argument_error_builds_nothing():
    W = wt()
    with pytest.raises(W.WTError) as e:
        W.build_batch([to_dev(np.zeros(10, np.uint8)), to_dev(np.zeros(10, np.uint8))], [4, 300])
    assert e.value.status == W.ERR_ARG


def test_large_batch_of_small_sequences():
    """Hundreds of short sequences in one call (many jobs per level launch)."""
    W = wt()
    specs = inputs.batch_specs(count=300, log2_min=8, log2_max=14)
    seqs = [sp.generate() for sp in specs]
    trees = W.build_batch([to_dev(S) for S in seqs], [sp.sigma for sp in specs])
    for sp, S, t in zip(specs, seqs, trees):
        compare_tree(t, S, sp.sigma, check_dir=False)


def test_batch_mid_alphabet_slabs():
    """Sequences with 8K..96K codes take the packed histogram in 1M-symbol
    slabs; a hot code passes the 2^15 hand-over inside one slab."""
    W = wt()
    seqs = [inputs.zipf((1 << 22) + 17, 65536, 1.3, 71, np.uint16), inputs.zipf(70_001, 20000, 1.1, 72, np.uint16),
            inputs.uniform(5000, 256, 73, np.uint8), inputs.zipf(1 << 20, 65536, 1.0, 74, np.uint32)]
    sigmas = [65536, 20000, 256, 65536]
    trees = W.build_batch([to_dev(S) for S in seqs], sigmas)
    for S, sigma, t in zip(seqs, sigmas, trees):
        compare_tree(t, S, sigma, check_dir=len(S) < (1 << 21))
