"""The seeded input generators on CPU: splitmix64 against its published first
outputs, the uniform and Zipf draws against their definitions (ranges,
frequencies, the seeded permutation of ranks), and the batched and serving
workloads against their stated shapes (length range, alphabets, widths,
distribution coin)."""
import math

import numpy as np
import pytest

from paper_1610_05994_gb300 import inputs


def test_splitmix64_published_first_outputs():
    # splitmix64 (Steele, Lea, Flood 2014) started from state 0: the first
    # three outputs of the reference generator.
    assert [int(v) for v in inputs.splitmix64(0, 0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                             0x06C45D188009454F]
    # Output start + k is independent of how the stream is cut.
    whole = inputs.splitmix64(12345, 0, 1000)
    assert np.array_equal(whole[300:700], inputs.splitmix64(12345, 300, 400))


@pytest.mark.parametrize("sigma", [1, 2, 4, 96, 256, 65536, 1 << 20])
def test_uniform_range_width_and_balance(sigma):
    n = 400_000
    S = inputs.uniform(n, sigma, 7)
    assert S.dtype == inputs.sym_dtype(sigma) and S.size == n
    assert int(S.max()) < sigma
    if sigma <= 256:
        counts = np.bincount(S, minlength=sigma)
        exp = n / sigma
        # Every code within 6 standard deviations of its expected count.
        assert np.all(np.abs(counts - exp) <= 6 * math.sqrt(exp) + 1)
    else:
        assert abs(S.mean() - (sigma - 1) / 2) < 0.01 * sigma


def test_uniform_multiply_shift_definition():
    # code = (top 32 bits of the stream) * sigma >> 32 (Lemire's reduction).
    s = inputs.splitmix64(99, 0, 1000)
    expect = ((s >> np.uint64(32)) * np.uint64(96)) >> np.uint64(32)
    assert np.array_equal(inputs.uniform(1000, 96, 99).astype(np.uint64), expect)


@pytest.mark.parametrize("sigma,alpha", [(96, 1.0), (256, 1.1), (65536, 1.0)])
def test_zipf_rank_frequencies_follow_the_law(sigma, alpha):
    n = 1_000_000
    S = inputs.zipf(n, sigma, alpha, 5)
    assert int(S.max()) < sigma
    perm = inputs.permutation(sigma, 5)
    assert np.array_equal(np.sort(perm), np.arange(sigma))  # a permutation of the codes
    counts = np.bincount(S, minlength=sigma)
    h = np.sum(np.arange(1, sigma + 1, dtype=np.float64) ** (-alpha))
    for r in range(4):  # rank r + 1 is code perm[r], with probability (r + 1)^-alpha / H
        p = (r + 1) ** (-alpha) / h
        assert abs(counts[perm[r]] - n * p) <= 6 * math.sqrt(n * p * (1 - p))
    # The most frequent code is the rank-1 code.
    assert int(np.argmax(counts)) == int(perm[0])


def test_named_workloads_shapes():
    w = inputs.WORKLOADS
    assert (w["u8-text-2^30-s96-zipf1.0"].n, w["u8-text-2^30-s96-zipf1.0"].sigma) == (1 << 30, 96)
    assert (w["u8-dna-2^30-s4"].n, w["u8-dna-2^30-s4"].sigma, w["u8-dna-2^30-s4"].dist) == (1 << 30, 4, "uniform")
    words = w["u32-words-2^29-s2^20-zipf1.2"]
    assert (words.n, words.sigma, words.width, words.alpha) == (1 << 29, 1 << 20, 4, 1.2)
    small = w["u8-uniform-2^20-s256"].generate()
    assert small.size == 1 << 20 and small.dtype == np.uint8
    # A prefix of a workload is the start of the whole sequence.
    t = w["u8-text-2^30-s96-zipf1.0"]
    assert np.array_equal(t.generate(1 << 16)[:1000], t.generate(1000))


def test_batch_specs_shape():
    specs = inputs.batch_specs()
    assert len(specs) == 4096
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 1 << 10 and ns.max() <= 1 << 22
    lg = np.log2(ns)
    assert abs(lg.mean() - 16.0) < 0.3            # log-uniform over [10, 22]
    assert abs(np.mean(lg < 16.0) - 0.5) < 0.05
    sig = [s.sigma for s in specs]
    for c in (4, 20, 256, 65536):
        assert abs(sig.count(c) / 4096 - 0.25) < 0.04
    assert all(s.width == (1 if s.sigma <= 256 else 2) for s in specs)
    zipfs = [s for s in specs if s.dist == "zipf"]
    assert abs(len(zipfs) / 4096 - 0.5) < 0.05 and all(s.alpha == 1.1 for s in zipfs)
    assert len({s.seed for s in specs}) == 4096
    assert specs[17] == inputs.batch_specs(count=32)[17]  # each spec depends only on its index


def test_serving_specs_shape():
    specs = inputs.serving_specs(2000)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 1 << 12 and ns.max() <= 1 << 26
    assert abs(np.log2(ns).mean() - 19.0) < 0.4   # log-uniform over [12, 26]
    assert {s.sigma for s in specs} == {256, 65536}
    assert all(s.dist == "zipf" and s.alpha == 1.0 for s in specs)
    assert all(s.width == (1 if s.sigma == 256 else 2) for s in specs)
