"""GPU parity of the wavelet matrix (wt_build_matrix_async): every bitmap
word, directory entry and count equals the oracle's matrix, and access, rank
and select on the GPU equal the oracle's matrix queries."""
import numpy as np
import pytest
import torch

from gpu_helpers import needs_gpu, query_batches, to_dev, tree_bits, wt
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def compare_matrix(m, S, sigma, queries=True):
    want = O.wm_bits(S, sigma)
    got = tree_bits(m)
    assert got.shape == want.shape
    n = len(S)
    for l in range(want.shape[0]):
        if not np.array_equal(got[l], want[l]):
            bad = np.flatnonzero(got[l] != want[l])
            raise AssertionError(f"level {l}: {len(bad)} bytes differ, first at byte {bad[0]}")
        lv = m.level(l)
        d = O.directory(want[l], n)
        assert np.array_equal(lv.R.cpu().numpy(), d["R"]), f"R level {l}"
        assert np.array_equal(lv.Hy.cpu().numpy(), d["Hy"]), f"Hy level {l}"
        assert np.array_equal(lv.S1.cpu().numpy(), d["S1"]), f"S1 level {l}"
        assert np.array_equal(lv.S0.cpu().numpy(), d["S0"]), f"S0 level {l}"
        assert lv.ones == d["ones"]
    if queries:
        I, Cs, J = query_batches(S, sigma, 3000, 17)
        Id, Cd, Jd = (torch.from_numpy(x).cuda() for x in (I, Cs, J))
        assert np.array_equal(m.access(Id).cpu().numpy(), O.wm_access(want, n, sigma, I))
        assert np.array_equal(m.rank(Cd, Id).cpu().numpy(), O.wm_rank(want, n, sigma, Cs, I))
        assert np.array_equal(m.select(Cd, Jd).cpu().numpy(), O.wm_select(want, n, sigma, Cs, J))
    return want


SIZES = [0, 1, 31, 33, 511, 512, 513, 8191, 8192, 8193, 16384, 65537, 100003]


@pytest.mark.parametrize("sigma", [1, 2, 3, 4, 5, 17, 96, 256])
@pytest.mark.parametrize("n", SIZES)
def test_matrix_bytes(sigma, n):
    W = wt()
    S = inputs.zipf(n, sigma, 1.0, 500 + n, np.uint8) if n else np.zeros(0, np.uint8)
    m = W.Tree.build(to_dev(S), sigma, matrix=True)
    info = m.info()
    assert info["layout"] == W.LAYOUT_MATRIX and info["levels"] == O.levels(sigma)
    compare_matrix(m, S, sigma, queries=n > 0)


@pytest.mark.parametrize("sigma,dtype,dist", [(1000, np.uint16, "uniform"), (65536, np.uint16, "zipf"),
                                              (4, np.uint32, "uniform"), ((1 << 20) + 3, np.uint32, "zipf")])
@pytest.mark.parametrize("n", [513, 8193, 70001])
def test_matrix_wide_codes(sigma, dtype, dist, n):
    W = wt()
    S = (inputs.zipf(n, sigma, 1.2, 7 + n, dtype) if dist == "zipf" else inputs.uniform(n, sigma, 7 + n, dtype))
    compare_matrix(W.Tree.build(to_dev(S), sigma, matrix=True), S, sigma)


def test_matrix_from_host_and_unaligned_device_input():
    W = wt()
    S = inputs.zipf(50001, 96, 1.0, 5, np.uint8)
    compare_matrix(W.Tree.build(S, 96, matrix=True), S, 96)
    D = to_dev(np.concatenate([np.zeros(3, np.uint8), S]))
    compare_matrix(W.Tree.build(D[3:], 96, matrix=True), S, 96)


def test_matrix_many_tiles():
    """Millions of symbols: every deep level mixes the top-bit keys in every tile."""
    W = wt()
    S = inputs.zipf(3_000_017, 4096, 1.2, 3, np.uint16)
    compare_matrix(W.Tree.build(to_dev(S), 4096, matrix=True), S, 4096, queries=True)


def test_matrix_of_text_at_2_24():
    W = wt()
    S = inputs.zipf(1 << 24, 96, 1.0, 11, np.uint8)
    compare_matrix(W.Tree.build(to_dev(S), 96, matrix=True), S, 96)


def test_matrix_and_tree_share_level_zero_and_the_answers():
    """Level 0 of both is the top-bit plane, and both answer the same queries."""
    W = wt()
    S = inputs.zipf(200003, 256, 1.1, 13, np.uint8)
    t = W.Tree.build(to_dev(S), 256)
    m = W.Tree.build(to_dev(S), 256, matrix=True)
    assert torch.equal(t.level(0).words, m.level(0).words)
    I, Cs, J = query_batches(S, 256, 4000, 19)
    Id, Cd, Jd = (torch.from_numpy(x).cuda() for x in (I, Cs, J))
    assert torch.equal(t.access(Id), m.access(Id))
    assert torch.equal(t.rank(Cd, Id), m.rank(Cd, Id))
    assert torch.equal(t.select(Cd, Jd), m.select(Cd, Jd))


def test_matrix_reports_symbols_out_of_range():
    W = wt()
    S = inputs.uniform(70000, 50, 3, np.uint8)
    S[12345] = 60
    with pytest.raises(W.WTError) as e:
        W.Tree.build(to_dev(S), 50, matrix=True)
    assert e.value.status == W.ERR_SYMBOL_RANGE


def test_multi_queries_and_merge_reject_matrices():
    W = wt()
    S = inputs.uniform(1000, 16, 1, np.uint8)
    m = W.Tree.build(to_dev(S), 16, matrix=True)
    t = W.Tree.build(to_dev(S), 16)
    z = torch.zeros(4, dtype=torch.uint32, device="cuda")
    with pytest.raises(W.WTError) as e:
        W.query_multi([t, m], z, z.to(torch.uint8), z, z.to(torch.uint64))
    assert e.value.status == W.ERR_ARG
    with pytest.raises(W.WTError) as e:
        W.merge([t, m])
    assert e.value.status == W.ERR_ARG
