"""GPU parity of construction: every bitmap word, directory entry and count of
trees built by the CUDA path through the C ABI equals the CPU oracle's."""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, to_dev, wt
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]

WORKLOAD_SMALL = inputs.WORKLOADS["u8-uniform-2^20-s256"]


VARIANTS = [1, 2, 3]  # one level per pass (kernels a+b+c), dd-direct (kernel d), two levels per pass


@pytest.mark.parametrize("variant", VARIANTS)
def test_small_workload_bit_exact(variant):
    """2^20 uniform bytes over 256 codes (8 levels): the full tree equals the oracle's."""
    W = wt()
    S = WORKLOAD_SMALL.generate()
    t = W.Tree.build(to_dev(S), WORKLOAD_SMALL.sigma, variant=variant)
    assert t.info()["variant"] == variant
    compare_tree(t, S, WORKLOAD_SMALL.sigma)


def test_auto_variant_is_a_concrete_variant_and_levelwise_for_wide_symbols():
    W = wt()
    a = W.Tree.build(to_dev(inputs.uniform(5000, 96, 1, np.uint8)), 96)
    b = W.Tree.build(to_dev(inputs.uniform(5000, 1000, 1, np.uint16)), 1000)
    c = W.Tree.build(to_dev(inputs.uniform(5000, 1000, 1, np.uint32)), 1000)
    assert a.info()["variant"] in (W.VARIANT_DD, W.VARIANT_PAIRS, W.VARIANT_LEVELWISE)
    assert b.info()["variant"] in (W.VARIANT_PAIRS, W.VARIANT_LEVELWISE)
    assert c.info()["variant"] == W.VARIANT_LEVELWISE


def test_dd_rejects_what_it_cannot_build():
    W = wt()
    with pytest.raises(W.WTError) as e:
        W.Tree.build(to_dev(inputs.uniform(100, 1000, 1, np.uint16)), 1000, variant=W.VARIANT_DD)
    assert e.value.status == W.ERR_ARG


SIZES = [0, 1, 31, 32, 33, 511, 512, 513, 2047, 2048, 2049, 4095, 4096, 4097, 8191, 8192, 8193, 16383, 16384, 16385,
         65535, 65537, 100003]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("sigma", [1, 2, 3, 4, 5, 16, 17, 96, 255, 256])
@pytest.mark.parametrize("n", SIZES)
def test_edge_shapes_u8(sigma, n, variant):
    W = wt()
    S = inputs.zipf(n, sigma, 1.0, 1000 + n, np.uint8) if n else np.zeros(0, np.uint8)
    if variant == W.VARIANT_DD and (sigma == 1 or n == 0):
        variant = W.VARIANT_AUTO  # nothing for dd to build
    t = W.Tree.build(to_dev(S), sigma, variant=variant)
    compare_tree(t, S, sigma)


@pytest.mark.parametrize("variant", [1, 3])
@pytest.mark.parametrize("sigma,dtype", [(257, np.uint16), (1000, np.uint16), (65536, np.uint16),
                                         (4, np.uint32), (1 << 20, np.uint32), ((1 << 20) + 3, np.uint32)])
@pytest.mark.parametrize("n", [1, 513, 2047, 2048, 2049, 4096, 4097, 70001])
def test_wide_symbols(sigma, dtype, n, variant):
    W = wt()
    S = inputs.zipf(n, sigma, 1.2, 77 + n, dtype)
    t = W.Tree.build(to_dev(S), sigma, variant=variant)
    compare_tree(t, S, sigma)


@pytest.mark.parametrize("n", [512, 1024, 4608, 8704, 65536 - 512, 65536])
def test_level0_count_with_a_partial_last_tile_on_reused_memory(n):
    """n a multiple of 512 (but not always of the 8192-symbol tile): every
    unit count the level step scans must be written by this build, also when
    its scratch reuses memory that held another build's counts (the big tree
    is freed in stream order just before, so its memory comes back)."""
    W = wt()
    big = to_dev(inputs.uniform(1 << 22, 256, 9, np.uint8))
    S = inputs.zipf(n, 96, 1.0, n, np.uint8)
    D = to_dev(S)
    for _ in range(3):
        W.Tree.build(big, 256, wait=False).free()
        t = W.Tree.build(D, 96, wait=False)
        t.wait()
        compare_tree(t, S, 96)


@pytest.mark.parametrize("variant", [1, 3])
def test_host_input_and_unaligned_device_input(variant):
    """S may be host memory; a device S that is not 16-byte aligned takes the scalar path."""
    W = wt()
    sigma = 96
    S = inputs.zipf(50001, sigma, 1.0, 5, np.uint8)
    compare_tree(W.Tree.build(S, sigma, variant=variant), S, sigma)
    D = to_dev(np.concatenate([np.zeros(3, np.uint8), S]))
    compare_tree(W.Tree.build(D[3:], sigma, variant=variant), S, sigma)
    S2 = inputs.zipf(70001, 1000, 1.1, 6, np.uint16)
    D2 = to_dev(np.concatenate([np.zeros(1, np.uint16), S2]))
    compare_tree(W.Tree.build(D2[1:], 1000, variant=variant), S2, 1000)


def test_many_tiles_zipf_multi_level_scatter():
    """Several thousand tiles, skewed codes: the look-back and the scatter stay exact."""
    W = wt()
    sigma = 1 << 12
    S = inputs.zipf(3_000_017, sigma, 1.2, 3, np.uint16)
    t = W.Tree.build(to_dev(S), sigma)
    compare_tree(t, S, sigma)


def test_symbol_out_of_range_is_reported():
    W = wt()
    S = np.array([0, 1, 2, 3, 4, 1], dtype=np.uint8)
    with pytest.raises(W.WTError) as e:
        W.Tree.build(to_dev(S), 4)
    assert e.value.status == W.ERR_SYMBOL_RANGE


@pytest.mark.parametrize("sigma,bad", [(3, 3), (4, 200), (96, 96)])
@pytest.mark.parametrize("n", [1 << 16, (1 << 16) + 5])
def test_symbol_out_of_range_in_long_byte_sequences(sigma, bad, n):
    """The bit-plane histogram (sigma <= 4) and the histogram that also counts
    level 0 (n a multiple of 512) flag a symbol >= sigma."""
    W = wt()
    S = inputs.uniform(n, sigma, 7, np.uint8)
    S[n // 3] = bad
    with pytest.raises(W.WTError) as e:
        W.Tree.build(to_dev(S), sigma)
    assert e.value.status == W.ERR_SYMBOL_RANGE


def test_invalid_arguments():
    W = wt()
    S = to_dev(np.zeros(10, np.uint8))
    for sigma in (0, 257):
        with pytest.raises(W.WTError) as e:
            W.Tree.build(S, sigma)
        assert e.value.status == W.ERR_ARG


def test_node_starts_stage():
    """Kernel (a): Hex equals the oracle's node starts."""
    W = wt()
    for sigma, dtype, n in ((256, np.uint8, 1 << 20), (96, np.uint8, 999_999), (4, np.uint8, 12345),
                            (65536, np.uint16, 300_001), (1 << 20, np.uint32, 200_003)):
        S = inputs.zipf(n, sigma, 1.0, 21, dtype)
        got = W.node_starts(to_dev(S), sigma).cpu().numpy()
        assert np.array_equal(got, O.node_starts(S, sigma)), sigma


def test_level_step_stage():
    """Kernels (b) + (c) one level at a time: bitmap and R of level l and the order P_{l+1}."""
    W = wt()
    for sigma, dtype, n in ((96, np.uint8, 100_003), (1 << 16, np.uint16, 70_001), (1 << 20, np.uint32, 50_000)):
        S = inputs.zipf(n, sigma, 1.1, 8, dtype)
        L = O.levels(sigma)
        hx = W.node_starts(to_dev(S), sigma)
        bits = O.build_bits(S, sigma)
        for l in range(L):
            P = O.level_order(S, sigma, l).astype(dtype)
            words, R, nxt = W.level_step(to_dev(P), sigma, l, hx, want_next=l + 1 < L)
            assert np.array_equal(words.cpu().numpy().view(np.uint8), bits[l]), (sigma, l)
            assert np.array_equal(R.cpu().numpy(), O.directory(bits[l], n)["R"]), (sigma, l)
            if l + 1 < L:
                assert np.array_equal(nxt.cpu().numpy(), O.level_order(S, sigma, l + 1).astype(dtype)), (sigma, l)


def test_async_build_on_stream_and_torch_allocator():
    W = wt()
    W.use_torch_allocator(True)
    try:
        sigma = 20
        S = inputs.uniform(200_001, sigma, 9, np.uint8)
        s = torch.cuda.Stream()
        D = to_dev(S)
        torch.cuda.synchronize()
        t = W.Tree.build(D, sigma, stream=s, wait=False)
        t.wait()
        compare_tree(t, S, sigma)
        t.free()
    finally:
        W.use_torch_allocator(False)


@pytest.mark.parametrize("matrix", [False, True])
def test_bitmaps_exact_over_memory_full_of_ones(matrix):
    """The passes write every bit of the level bitmaps they hand over (whole
    words by stores, words shared by runs by clearing and setting their own
    bits) and the padding is zeroed: built in memory that held all-ones bytes
    (torch's caching allocator hands the library a block just filled with
    0xFF), every level still equals the oracle's, padding included."""
    W = wt()
    W.use_torch_allocator(True)
    try:
        cases = [(96, inputs.zipf(3 * 8192 * 7 + 12345, 96, 1.0, 3), np.uint8),
                 (4, inputs.uniform(100_003, 4, 4, np.uint8), np.uint8),
                 (65536, inputs.zipf(200_001, 65536, 1.1, 5).astype(np.uint16), np.uint16),
                 (1000, inputs.zipf((1 << 18) + 33, 1000, 1.0, 6).astype(np.uint16), np.uint16)]
        for sigma, S, dtype in cases:
            for variant in ([1] if matrix else [1, 3]):
                junk = torch.full((64 << 20,), 255, dtype=torch.uint8, device="cuda")
                del junk  # back to the cache, still holding the ones
                D = to_dev(S.astype(dtype))
                t = W.Tree.build(D, sigma, variant=variant, matrix=matrix)
                if matrix:
                    want = O.wm_bits(S, sigma)
                    for l in range(want.shape[0]):
                        assert np.array_equal(t.level(l).words.cpu().numpy().view(np.uint8), want[l]), (sigma, l)
                else:
                    compare_tree(t, S, sigma)
                t.free()
                del D
    finally:
        W.use_torch_allocator(False)


@pytest.mark.parametrize("sigma,dtype,log2n,alpha,variant", [
    (96, np.uint8, 25, 1.0, 1), (4, np.uint8, 25, 0.0, 1), (96, np.uint8, 25, 1.0, 2), (4, np.uint8, 25, 0.0, 2),
    (256, np.uint8, 24, 0.0, 2), (65536, np.uint16, 23, 1.1, 1), (1 << 20, np.uint32, 22, 1.2, 1),
    (96, np.uint8, 25, 1.0, 3), (4, np.uint8, 25, 0.0, 3), (256, np.uint8, 24, 0.0, 3), (20, np.uint8, 24, 1.1, 3),
    (16, np.uint8, 25, 0.0, 3), (65536, np.uint16, 23, 1.1, 3), (4096, np.uint16, 24, 1.2, 3)])
def test_many_tiles_per_cta_pipeline(sigma, dtype, log2n, alpha, variant):
    """Enough tiles that every persistent CTA streams several (the producer /
    compute pipeline runs at full depth), plus a ragged tail."""
    W = wt()
    n = (1 << log2n) + 777
    S = inputs.zipf(n, sigma, alpha, 4242, dtype) if alpha else inputs.uniform(n, sigma, 4242, dtype)
    t = W.Tree.build(to_dev(S), sigma, variant=variant)
    compare_tree(t, S, sigma)


@pytest.mark.parametrize("sigma,dtype,n", [(65536, np.uint16, 1 << 25), (98304, np.uint32, 300_001),
                                           (49153, np.uint16, 1_000_003)])
def test_mid_alphabet_histogram(sigma, dtype, n):
    """Alphabets of 48K..96K codes use packed 16-bit shared bins; a skewed
    sequence drives its hottest bin past the 2^15 hand-over many times."""
    W = wt()
    S = inputs.zipf(n, sigma, 1.3, 901 + sigma, dtype)
    t = W.Tree.build(to_dev(S), sigma, variant=W.VARIANT_LEVELWISE)
    starts = W.node_starts(to_dev(S), sigma).cpu().numpy()
    L = (sigma - 1).bit_length()
    want = np.zeros((1 << L) + 1, np.uint64)
    want[1:sigma + 1] = np.cumsum(np.bincount(S, minlength=sigma)).astype(np.uint64)
    want[sigma + 1:] = n
    assert np.array_equal(starts, want)
    compare_tree(t, S, sigma, check_dir=n < (1 << 24))


@pytest.mark.parametrize("sigma", [(1 << 20) + 3, 100_000, (1 << 22)])
def test_large_alphabets_at_millions_of_symbols(sigma):
    """Four-byte codes over large alphabets (the replicated global histogram,
    deep levels of tiny nodes) at n > 2^22: whole trees equal the oracle's."""
    W = wt()
    n = (1 << 22) + 12345
    S = inputs.zipf(n, sigma, 1.2, 4242, np.uint32)
    t = W.Tree.build(to_dev(S), sigma)
    compare_tree(t, S, sigma)
    t.free()


def test_large_alphabet_flags_out_of_range_symbols():
    W = wt()
    sigma = (1 << 20) + 3
    S = inputs.zipf((1 << 22) + 7, sigma, 1.2, 99, np.uint32)
    S[123457] = sigma
    with pytest.raises(W.WTError) as e:
        W.Tree.build(to_dev(S), sigma)
    assert e.value.status == W.ERR_SYMBOL_RANGE


@pytest.mark.parametrize("sigma,dtype,log2n,want", [
    (96, np.uint8, 20, "dd"), (4, np.uint8, 20, "dd"), (4, np.uint8, 22, "levelwise"),
    (96, np.uint8, 25, "levelwise"), (1000, np.uint16, 20, "pairs"), (1000, np.uint16, 23, "levelwise"),
    (65536, np.uint16, 18, "levelwise"), (1 << 20, np.uint32, 18, "levelwise")])
def test_auto_follows_the_measured_table_and_is_bit_exact(sigma, dtype, log2n, want):
    """The autotuner's choice (the measured table of choose_variant) for a few
    (width, levels, n) entries, and the tree it builds equals the oracle's."""
    W = wt()
    n = (1 << log2n) - 3
    S = inputs.zipf(n, sigma, 1.0, 600 + log2n, dtype)
    t = W.Tree.build(to_dev(S), sigma)
    names = {W.VARIANT_LEVELWISE: "levelwise", W.VARIANT_DD: "dd", W.VARIANT_PAIRS: "pairs"}
    assert names[t.info()["variant"]] == want
    compare_tree(t, S, sigma)
