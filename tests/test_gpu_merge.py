"""GPU parity of the merge of partial trees (the buffered build of Section 5,
merged with Algorithm 2's global offsets and Function mergeBA): the merged
tree's bitmaps, directories and counts equal the oracle's tree of the
concatenation, and the oracle's own merge of the same parts."""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, query_batches, to_dev, wt
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def parts_of(cuts, sigma, seed, dist="uniform"):
    dt = inputs.sym_dtype(sigma)
    out = []
    for i, c in enumerate(cuts):
        if dist == "zipf":
            out.append(inputs.zipf(c, sigma, 1.1, seed + i, dt))
        else:
            out.append(inputs.uniform(c, sigma, seed + i, dt))
    return out


def check_merge(W, parts, sigma, trees=None, queries=True):
    trees = trees or [W.Tree.build(to_dev(p), sigma) for p in parts]
    m = W.merge(trees)
    S = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    assert m.n == len(S)
    want = compare_tree(m, S, sigma)
    # The oracle's merge of the same parts gives the same bitmaps.
    if parts and O.levels(sigma):
        om = O.merge_bits([O.build_bits(p, sigma) for p in parts], [len(p) for p in parts],
                          [O.node_starts(p, sigma) for p in parts], sigma)
        assert np.array_equal(om, want)
    if queries and len(S):
        I, Cs, J = query_batches(S, sigma, 2000, 5)
        assert np.array_equal(m.access(torch.from_numpy(I).cuda()).cpu().numpy(), O.access(want, len(S), sigma, I))
        assert np.array_equal(m.rank(torch.from_numpy(Cs).cuda(), torch.from_numpy(I).cuda()).cpu().numpy(),
                              O.rank(want, len(S), sigma, Cs, I))
        assert np.array_equal(m.select(torch.from_numpy(Cs).cuda(), torch.from_numpy(J).cuda()).cpu().numpy(),
                              O.select(want, len(S), sigma, Cs, J))
    return m


CUTS = [
    [100000],
    [0, 5000],
    [1, 31, 33, 511, 513],
    [4097, 0, 8191, 65537, 3],
    [131072, 131072],
    [70001, 1, 99999],
]


@pytest.mark.parametrize("sigma", [2, 4, 5, 96, 256])
@pytest.mark.parametrize("cuts", CUTS)
def test_merge_bytes(sigma, cuts):
    """1-byte codes, ragged parts (empty, single symbol, word and block edges)."""
    W = wt()
    check_merge(W, parts_of(cuts, sigma, 11), sigma)


@pytest.mark.parametrize("sigma,dist", [(1000, "uniform"), (65536, "zipf"), ((1 << 20) + 3, "zipf")])
def test_merge_wide_codes(sigma, dist):
    """2- and 4-byte codes, up to 21 levels with mostly empty deep nodes."""
    W = wt()
    check_merge(W, parts_of([40000, 17, 90001, 2048], sigma, 23, dist), sigma)


def test_merge_of_many_small_parts():
    """64 parts of 0..3000 symbols: most output words take bits of several runs."""
    W = wt()
    rng = np.random.default_rng(3)
    cuts = [int(x) for x in rng.integers(0, 3000, 64)]
    cuts[5] = 0
    check_merge(W, parts_of(cuts, 256, 31, "zipf"), 256)


def test_merge_of_parts_on_disjoint_alphabet_halves():
    """Every node of the result is empty in some part."""
    W = wt()
    a = inputs.uniform(30000, 32, 1, np.uint8)
    b = (inputs.uniform(50000, 32, 2, np.uint8) + 32).astype(np.uint8)
    c = inputs.uniform(7777, 64, 3, np.uint8)
    check_merge(W, [a, b, c], 64)


def test_merge_of_one_part_is_a_copy():
    W = wt()
    S = inputs.zipf(123457, 96, 1.0, 4, np.uint8)
    check_merge(W, [S], 96)


def test_merge_of_empty_parts():
    W = wt()
    parts = [np.zeros(0, np.uint8), np.zeros(0, np.uint8)]
    m = check_merge(W, parts, 20)
    assert m.info()["n"] == 0


def test_merge_sigma_one():
    W = wt()
    parts = [np.zeros(1000, np.uint8), np.zeros(3, np.uint8)]
    m = W.merge([W.Tree.build(to_dev(p), 1) for p in parts])
    assert m.info()["levels"] == 0 and m.n == 1003
    r = m.rank(torch.zeros(2, dtype=torch.uint32, device="cuda"), torch.tensor([0, 1003], device="cuda"))
    assert r.cpu().tolist() == [0, 1003]


@pytest.mark.parametrize("variant", [1, 2])
def test_merge_of_parts_built_by_either_variant(variant):
    W = wt()
    parts = parts_of([50000, 20001], 16, 41)
    trees = [W.Tree.build(to_dev(p), 16, variant=variant) for p in parts]
    check_merge(W, parts, 16, trees=trees)


def test_merge_of_batch_built_parts():
    W = wt()
    parts = parts_of([3000, 0, 10000, 777], 200, 51, "zipf")
    trees = W.build_batch([to_dev(p) for p in parts], [200] * len(parts))
    check_merge(W, parts, 200, trees=trees)


def test_merge_on_a_side_stream():
    W = wt()
    parts = parts_of([9000, 12000], 96, 61)
    trees = [W.Tree.build(to_dev(p), 96) for p in parts]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m = W.merge(trees, stream=s)
    compare_tree(m, np.concatenate(parts), 96)


def test_merge_rejects_mixed_alphabets_and_widths():
    W = wt()
    a = W.Tree.build(to_dev(inputs.uniform(100, 4, 1, np.uint8)), 4)
    b = W.Tree.build(to_dev(inputs.uniform(100, 8, 2, np.uint8)), 8)
    c = W.Tree.build(to_dev(inputs.uniform(100, 4, 3, np.uint16)), 4)
    for bad in ([a, b], [a, c]):
        with pytest.raises(W.WTError) as e:
            W.merge(bad)
        assert e.value.status == W.ERR_ARG
    with pytest.raises(W.WTError):
        W.merge([])


@pytest.mark.parametrize("n,chunk", [(200000, 12345), (100000, 100000), (100000, 1 << 20), (50, 1), (65536, 512)])
def test_chunked_build_from_host_and_device(n, chunk):
    """Section 5's buffered build: chunks built alone, then merged."""
    W = wt()
    S = inputs.zipf(n, 96, 1.0, 71, np.uint8)
    compare_tree(W.build_chunked(S, 96, chunk), S, 96)
    compare_tree(W.build_chunked(to_dev(S), 96, chunk), S, 96)


def test_chunked_build_wide_codes():
    W = wt()
    S = inputs.zipf(300001, 70000, 1.2, 73, np.uint32)
    compare_tree(W.build_chunked(S, 70000, 65536), S, 70000)


def test_chunked_build_reports_symbols_out_of_range():
    W = wt()
    S = inputs.uniform(100000, 50, 75, np.uint8)
    S[77777] = 50
    with pytest.raises(W.WTError) as e:
        W.build_chunked(S, 50, 10000)
    assert e.value.status == W.ERR_SYMBOL_RANGE
    with pytest.raises(W.WTError) as e:
        W.build_chunked(S, 50, 0)
    assert e.value.status == W.ERR_ARG


def test_chunked_build_of_text_at_2_26():
    """2^26 Zipf text symbols in 2^24-symbol chunks: four partial trees merged."""
    W = wt()
    S = inputs.zipf(1 << 26, 96, 1.0, 77, np.uint8)
    compare_tree(W.build_chunked(S, 96, 1 << 24), S, 96)
