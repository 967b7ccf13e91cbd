"""Pins for the CPU oracle: checks against what the paper prints, closed forms,
library routines and brute force, never against the oracle's own formulas.

Each test names the part of the oracle a plausible mistake would break:
a dropped term, a wrong bit index, an off-by-one rank, a transposed loop.
"""
import itertools

import numpy as np
import pytest

from conftest import read_golden
from oracle import oracle as O
from paper_1610_05994_gb300 import inputs


def unpack(level_row, n):
    """Bits 0..n-1 of one level (bit p at byte p>>3, bit p&7)."""
    return np.unpackbits(level_row, bitorder="little")[:n]


def stable_level_order(S, sigma, l):
    """P_l by numpy's stable sort on the key s >> (L-l) (a library routine)."""
    L = O.levels(sigma)
    key = S.astype(np.uint64) >> np.uint64(L - l)
    return S[np.argsort(key, kind="stable")]


# ---------------------------------------------------------------- worked example

def example():
    g = read_golden("worked_example.txt")
    alphabet = g["alphabet"].split(",")
    code = {ch: i for i, ch in enumerate(alphabet)}
    S = np.array([code[ch] for ch in g["sequence"]], dtype=np.uint8)
    return g, alphabet, S


def test_worked_example_access_and_trace():
    """Section 2.2: access(S, 24) = 't' with in-node indices 7, 4, 2 (Fig. 2)."""
    g, alphabet, S = example()
    sigma = len(alphabet)
    assert sigma == 16 and O.levels(sigma) == 4 and len(S) == 30
    bits = O.build_bits(S, sigma)
    i = int(g["access_index"])
    sym, trace = O.access_trace(bits, len(S), sigma, i)
    assert sym == int(g["access_code"])
    assert alphabet[sym] == g["access_symbol"]
    want = [int(v) for v in g["trace"].split(",")]
    assert trace[:3] == want
    # The leaf is a single symbol: the index inside it is its rank among equal symbols.
    assert trace[3] == int(np.sum(S[:i] == sym))
    # The root bit read at position 24 is the first walked bit (a 1: go right).
    assert (int(bits[0, i >> 3]) >> (i & 7)) & 1 == int(g["bits"].split(",")[0])


def test_worked_example_levels_visit_expected_bits():
    """The walk of Section 2.2 reads bits 1,0,0,0 (right, left, left, left)."""
    g, alphabet, S = example()
    sigma = len(alphabet)
    bits = O.build_bits(S, sigma)
    i = int(g["access_index"])
    sym, trace = O.access_trace(bits, len(S), sigma, i)
    assert [(sym >> (3 - l)) & 1 for l in range(4)] == [int(b) for b in g["bits"].split(",")]


def test_worked_example_fig3_positions():
    """The caption of Fig. 3 names S[10]='a', S[15]='e', S[19]='P', S[26]='d'."""
    g, alphabet, S = example()
    bits = O.build_bits(S, len(alphabet))
    for item in g["symbol_at"].split(","):
        pos, ch = item.split(":")
        assert alphabet[int(O.access(bits, len(S), 16, [int(pos)])[0])] == ch


# ---------------------------------------------------------------- construction

def test_level_zero_is_msb_plane():
    """Level 0 holds the most significant bit of every symbol in S order."""
    rng = np.random.default_rng(1)
    for sigma in (2, 3, 7, 96, 256):
        S = rng.integers(0, sigma, 3001).astype(np.uint8)
        L = O.levels(sigma)
        bits = O.build_bits(S, sigma)
        assert np.array_equal(unpack(bits[0], len(S)), (S >> (L - 1)) & 1)


def test_sigma_two_level_is_the_sequence():
    S = np.random.default_rng(2).integers(0, 2, 777).astype(np.uint8)
    bits = O.build_bits(S, 2)
    assert bits.shape[0] == 1
    assert np.array_equal(unpack(bits[0], len(S)), S)


@pytest.mark.parametrize("sigma,n,width", [(4, 1000, 1), (20, 2049, 1), (96, 5000, 1), (256, 4097, 1),
                                           (1000, 3000, 2), (65536, 2000, 2), (1 << 20, 1500, 4)])
def test_level_orders_are_stable_sorts(sigma, n, width):
    """P_l equals S stably sorted by the top l bits (Shun's sortWT view, Section 2.2)."""
    dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[width]
    S = inputs.zipf(n, sigma, 1.1, 7, dt)
    L = O.levels(sigma)
    for l in range(L + 1):
        assert np.array_equal(O.level_order(S, sigma, l), stable_level_order(S, sigma, l).astype(np.uint32))
    # The leaf order is the plain stable sort of S.
    assert np.array_equal(O.level_order(S, sigma, L), np.sort(S, kind="stable").astype(np.uint32))


@pytest.mark.parametrize("sigma", [3, 4, 5, 20, 96, 256, 300, 65536])
def test_bitmaps_from_library_sort(sigma):
    """B_l[p] = bit L-1-l of the stably sorted sequence; padding bits are zero."""
    rng = np.random.default_rng(sigma)
    n = 4999
    S = rng.integers(0, sigma, n).astype(inputs.sym_dtype(sigma))
    L = O.levels(sigma)
    bits = O.build_bits(S, sigma)
    assert bits.shape == (L, ((n + 511) // 512) * 64)
    for l in range(L):
        P = stable_level_order(S, sigma, l).astype(np.uint64)
        want = ((P >> np.uint64(L - 1 - l)) & np.uint64(1)).astype(np.uint8)
        full = np.unpackbits(bits[l], bitorder="little")
        assert np.array_equal(full[:n], want)
        assert not full[n:].any()


@pytest.mark.parametrize("sigma", [2, 4, 20, 96, 256, 1000])
def test_ones_per_level_match_histogram(sigma):
    """Ones on level l = sum over codes c of H[c] * bit l of c; node sizes = histogram sums."""
    S = inputs.zipf(6000, sigma, 1.0, 11, inputs.sym_dtype(sigma))
    L = O.levels(sigma)
    H = np.bincount(S, minlength=sigma)
    bits = O.build_bits(S, sigma)
    codes = np.arange(sigma)
    for l in range(L):
        ones = int(unpack(bits[l], len(S)).sum())
        assert ones == int((H * ((codes >> (L - 1 - l)) & 1)).sum())
        # node v of level l is the contiguous run of P_l with key v, of size sum of H over the node
        P = O.level_order(S, sigma, l)
        keys = P >> (L - l)
        sizes = np.bincount(keys, minlength=1 << l)
        want = np.bincount(codes >> (L - l), weights=H, minlength=1 << l).astype(np.int64)
        assert np.array_equal(sizes, want)
        assert np.all(np.diff(keys.astype(np.int64)) >= 0)


@pytest.mark.parametrize("sigma", [2, 3, 5, 16, 96, 256, 4096])
def test_algorithm1_and_dd_agree_with_definition(sigma):
    """Algorithm 1 (pwt) and Algorithm 2 (dd, several k) give the defined bitmaps."""
    S = inputs.uniform(3333, sigma, 5, inputs.sym_dtype(sigma))
    want = O.build_bits(S, sigma)
    assert np.array_equal(O.pwt_bits(S, sigma), want)
    for k in (1, 2, 3, 7, 64):
        assert np.array_equal(O.dd_bits(S, sigma, k), want), k


@pytest.mark.parametrize("sigma", [2, 3, 16, 96, 65536, (1 << 20) + 3])
def test_algorithm1_single_level_equals_library_sort(sigma):
    """Level l alone (Algorithm 1's per-level body) is bit L-1-l of S stably
    sorted by its top l bits, padding zero, for every l; out-of-range level
    and symbol are errors."""
    rng = np.random.default_rng(sigma + 3)
    n = 5003
    S = rng.integers(0, sigma, n).astype(inputs.sym_dtype(sigma))
    L = O.levels(sigma)
    for l in range(L):
        P = stable_level_order(S, sigma, l).astype(np.uint64)
        want = ((P >> np.uint64(L - 1 - l)) & np.uint64(1)).astype(np.uint8)
        full = np.unpackbits(O.pwt_level_bits(S, sigma, l), bitorder="little")
        assert np.array_equal(full[:n], want), l
        assert not full[n:].any()
    with pytest.raises(O.OracleError):
        O.pwt_level_bits(S, sigma, L)
    bad = S.copy()
    bad[7] = sigma if sigma < (1 << (8 * bad.itemsize)) else 0
    if bad[7] == sigma:
        with pytest.raises(O.OracleError):
            O.pwt_level_bits(bad, sigma, 0)


def test_sigma_one_has_no_levels():
    S = np.zeros(100, dtype=np.uint8)
    assert O.levels(1) == 0
    assert O.build_bits(S, 1).shape == (0, 64)
    assert list(O.access(np.zeros((0, 64), np.uint8), 100, 1, [0, 99, 100])) == [0, 0, 0xFFFFFFFF]
    assert list(O.rank(np.zeros((0, 64), np.uint8), 100, 1, [0, 0, 1], [5, 100, 3])) == [5, 100, 2**64 - 1]
    assert list(O.select(np.zeros((0, 64), np.uint8), 100, 1, [0, 0, 0], [1, 100, 101])) == [0, 99, 2**64 - 1]


def test_symbol_out_of_range_is_an_error():
    with pytest.raises(O.OracleError):
        O.build_bits(np.array([0, 1, 4], dtype=np.uint8), 4)


# ---------------------------------------------------------------- queries by brute force

def brute_check(S, sigma):
    n = len(S)
    bits = O.build_bits(S, sigma)
    I = np.arange(n + 1, dtype=np.uint64)
    acc = O.access(bits, n, sigma, I)
    assert np.array_equal(acc[:n], S.astype(np.uint32))
    assert acc[n] == 0xFFFFFFFF
    for c in range(sigma + 1):
        r = O.rank(bits, n, sigma, np.full(n + 2, c), np.arange(n + 2))
        for i in range(n + 2):
            if c >= sigma or i > n:
                assert r[i] == 2**64 - 1
            else:
                assert r[i] == int(np.sum(S[:i] == c))
        occ = np.flatnonzero(S == c)
        j = np.arange(len(occ) + 2)
        s = O.select(bits, n, sigma, np.full(len(j), c), j)
        for jj in j:
            if c >= sigma or jj == 0 or jj > len(occ):
                assert s[jj] == 2**64 - 1
            else:
                assert s[jj] == occ[jj - 1]


def test_queries_exhaustive_tiny():
    """access, rank, select on every sequence over sigma <= 4 with n <= 5."""
    for sigma in (1, 2, 3, 4):
        for n in range(0, 6 if sigma < 4 else 5):
            for t in itertools.product(range(sigma), repeat=n):
                brute_check(np.array(t, dtype=np.uint8), sigma)


@pytest.mark.parametrize("sigma,n", [(5, 200), (17, 300), (64, 257), (256, 513), (1000, 700)])
def test_queries_random(sigma, n):
    S = np.random.default_rng(sigma * n).integers(0, sigma, n).astype(inputs.sym_dtype(sigma))
    brute_check(S, sigma)


def test_select_inverts_rank():
    """select_c(rank_c(i) + 1) = i whenever S[i] = c."""
    sigma = 96
    S = inputs.zipf(20000, sigma, 1.0, 3, np.uint8)
    n = len(S)
    bits = O.build_bits(S, sigma)
    I = np.arange(0, n, 7, dtype=np.uint64)
    c = S[I.astype(np.int64)].astype(np.uint32)
    r = O.rank(bits, n, sigma, c, I)
    assert np.array_equal(O.select(bits, n, sigma, c, r + 1), I)


def test_level_symbol_matches_level_order():
    """Single-position sampling from the definition agrees with the full partition."""
    sigma = 40
    S = inputs.zipf(2500, sigma, 1.0, 9, np.uint8)
    L = O.levels(sigma)
    for l in range(L):
        P = O.level_order(S, sigma, l)
        for p in (0, 1, 777, 1249, 2499):
            assert O.level_symbol(S, sigma, l, p) == P[p]


# ---------------------------------------------------------------- directory

def test_directory_against_cumsum():
    """R, Hy, S1, S0 as recomputed with numpy's cumulative sums of the bits."""
    rng = np.random.default_rng(4)
    for n in (0, 1, 511, 512, 513, 8191, 8192, 8193, 100000):
        bits = rng.integers(0, 2, n).astype(np.uint8)
        row = np.packbits(np.concatenate([bits, np.zeros((-n) % 512, np.uint8)]), bitorder="little")
        d = O.directory(row, n)
        cs = np.concatenate([[0], np.cumsum(bits, dtype=np.uint64)])
        nb = (n + 511) // 512
        assert np.array_equal(d["R"], (cs[np.minimum(np.arange(nb + 1) * 512, n)] % (1 << 32)).astype(np.uint32))
        assert list(d["Hy"]) == [0, int(cs[n])] if n else list(d["Hy"]) == [0]
        ones_pos = np.flatnonzero(bits)
        zero_pos = np.flatnonzero(bits == 0)
        assert np.array_equal(d["S1"], (ones_pos[::8192] >> 9).astype(np.uint32))
        assert np.array_equal(d["S0"], (zero_pos[::8192] >> 9).astype(np.uint32))
        assert d["ones"] == int(cs[n])


def test_directory_closed_forms():
    """All-ones, all-zeros and alternating bitmaps have closed-form entries."""
    n = 3 * 8192 + 100
    nb = (n + 511) // 512
    ones = np.full(nb * 64, 0xFF, np.uint8)
    d = O.directory(ones, n)
    assert list(d["R"][:-1]) == [512 * b for b in range(nb)] and d["R"][-1] == n
    assert list(d["S1"]) == [16 * k for k in range(4)] and len(d["S0"]) == 0
    zeros = np.zeros(nb * 64, np.uint8)
    d = O.directory(zeros, n)
    assert not d["R"].any() and list(d["S0"]) == [16 * k for k in range(4)]
    alt = np.full(nb * 64, 0x55, np.uint8)   # bits 0,2,4,... set
    d = O.directory(alt, n)
    assert list(d["R"][:-1]) == [256 * b for b in range(nb)]
    assert list(d["S1"]) == [(2 * 8192 * k) >> 9 for k in range(2)]


@pytest.mark.slow
def test_directory_beyond_2_32_bits():
    """Past 2^32 bits the u32 block counts wrap while the hyper entries stay exact."""
    n = (1 << 32) + 1000
    nb = (n + 511) // 512
    row = np.full(nb * 64, 0xFF, np.uint8)
    d = O.directory(row, n)
    b = np.arange(nb + 1, dtype=np.uint64)
    want = np.minimum(b * np.uint64(512), np.uint64(n)) % np.uint64(1 << 32)
    assert np.array_equal(d["R"], want.astype(np.uint32))
    assert list(d["Hy"]) == [0, 1 << 32, n]
    assert d["ones"] == n and len(d["S1"]) == (n + 8191) // 8192


@pytest.mark.parametrize("sigma", [1, 2, 3, 20, 96, 256, 1000])
def test_node_starts_are_histogram_prefix(sigma):
    """Hex from numpy's bincount and cumsum; node v of level l starts at Hex[v << (L-l)]."""
    S = inputs.zipf(5000, sigma, 1.0, 13, inputs.sym_dtype(sigma))
    L = O.levels(sigma)
    H = np.bincount(S, minlength=1 << L)
    want = np.concatenate([[0], np.cumsum(H)]).astype(np.uint64)
    hx = O.node_starts(S, sigma)
    assert np.array_equal(hx, want)
    for l in range(L):
        keys = O.level_order(S, sigma, l) >> (L - l)
        for v in range(1 << l):
            hits = np.flatnonzero(keys == v)
            if len(hits):
                assert hits[0] == hx[v << (L - l)]


# ---------------------------------------------------------------- merge of partial trees

def sorted_bits(S, sigma):
    """Level bitmaps of S from numpy's stable sort (a library routine), padded."""
    L = O.levels(sigma)
    n = len(S)
    out = np.zeros((L, ((n + 511) // 512) * 64), dtype=np.uint8)
    for l in range(L):
        P = stable_level_order(S, sigma, l).astype(np.uint64)
        b = ((P >> np.uint64(L - 1 - l)) & np.uint64(1)).astype(np.uint8)
        b = np.concatenate([b, np.zeros(out.shape[1] * 8 - n, np.uint8)])
        out[l] = np.packbits(b, bitorder="little")
    return out


def hist_starts(S, sigma):
    """Node starts of S from numpy's bincount and cumsum."""
    H = np.bincount(S, minlength=1 << O.levels(sigma))
    return np.concatenate([[0], np.cumsum(H)]).astype(np.uint64)


@pytest.mark.parametrize("sigma", [1, 2, 5, 20, 96, 256, 300, 65536])
@pytest.mark.parametrize("cuts", [[0], [777], [0, 0], [300, 0, 700], [1, 1, 1, 1, 1], [513, 2000, 0, 37, 4096]])
def test_merge_of_partial_trees_is_the_tree_of_the_concatenation(sigma, cuts):
    """Merging the parts' trees (Section 5, Algorithm 2's offsets, mergeBA)
    gives the tree of S_0 S_1 ... S_{k-1}: compared with numpy's stable sort of
    the concatenation.  Parts and node starts come from numpy too, so a
    part-major copy order, a dropped part or a shifted offset fails here."""
    rng = np.random.default_rng(sigma + len(cuts))
    dt = inputs.sym_dtype(sigma)
    parts = [rng.integers(0, sigma, c).astype(dt) for c in cuts]
    merged = O.merge_bits([sorted_bits(p, sigma) for p in parts], cuts, [hist_starts(p, sigma) for p in parts],
                          sigma)
    S = np.concatenate(parts)
    assert np.array_equal(merged, sorted_bits(S, sigma))


def test_merge_of_skewed_parts_with_empty_nodes():
    """Parts drawn from disjoint halves of the alphabet: every node of the
    result is empty in some part, so the node-major order is visible."""
    sigma = 64
    a = np.arange(0, 32, dtype=np.uint8).repeat(5)
    b = np.arange(32, 64, dtype=np.uint8)[::-1].repeat(3)
    c = np.array([63, 0, 31, 32] * 50, dtype=np.uint8)
    parts = [a, b, c]
    merged = O.merge_bits([sorted_bits(p, sigma) for p in parts], [len(p) for p in parts],
                          [hist_starts(p, sigma) for p in parts], sigma)
    assert np.array_equal(merged, sorted_bits(np.concatenate(parts), sigma))


def test_merge_of_worked_example_in_three_parts():
    """The worked example of Section 2.2 cut into three parts (as in the dd
    example of Section 3.2) and merged answers the paper's access(S, 24)."""
    g, alphabet, S = example()
    sigma = len(alphabet)
    parts = [S[:10], S[10:21], S[21:]]
    merged = O.merge_bits([sorted_bits(p, sigma) for p in parts], [len(p) for p in parts],
                          [hist_starts(p, sigma) for p in parts], sigma)
    i = int(g["access_index"])
    assert int(O.access(merged, len(S), sigma, [i])[0]) == int(g["access_code"])
    assert alphabet[int(O.access(merged, len(S), sigma, [i])[0])] == g["access_symbol"]
    assert list(O.access(merged, len(S), sigma, np.arange(len(S)))) == list(S)


def test_merge_rejects_inconsistent_node_starts():
    S = np.array([0, 1, 2, 3], dtype=np.uint8)
    hx = hist_starts(S, 4)
    hx[-1] = 5  # does not end at the part's length
    with pytest.raises(O.OracleError):
        O.merge_bits([sorted_bits(S, 4)], [4], [hx], 4)


# ---------------------------------------------------------------- wavelet matrix

def wm_order(S, sigma, l):
    """S_l of the wavelet matrix by numpy's stable sort on the reversed top l
    bits (the last partition bit is the most significant key)."""
    L = O.levels(sigma)
    x = S.astype(np.uint64)
    key = np.zeros(len(S), np.uint64)
    for t in range(l):
        key |= ((x >> np.uint64(L - 1 - t)) & np.uint64(1)) << np.uint64(t)
    return S[np.argsort(key, kind="stable")]


@pytest.mark.parametrize("sigma", [2, 3, 4, 5, 20, 96, 256, 300, 65536, (1 << 20) + 3])
def test_matrix_levels_from_library_sort(sigma):
    """B_l[p] = bit L-1-l of S_l, S_l from numpy's stable argsort; padding zero."""
    rng = np.random.default_rng(sigma)
    n = 3001
    S = rng.integers(0, sigma, n).astype(inputs.sym_dtype(sigma))
    L = O.levels(sigma)
    bits = O.wm_bits(S, sigma)
    assert bits.shape == (L, ((n + 511) // 512) * 64)
    for l in range(L):
        P = wm_order(S, sigma, l).astype(np.uint64)
        want = ((P >> np.uint64(L - 1 - l)) & np.uint64(1)).astype(np.uint8)
        full = np.unpackbits(bits[l], bitorder="little")
        assert np.array_equal(full[:n], want), l
        assert not full[n:].any()


def test_matrix_small_worked_case():
    """S = 3 0 2 1 3 3 0 over 4 codes, by hand: level 0 holds the high bits
    1010110; S_1 = 0 1 0 3 2 3 3 (zeros of level 0 first) holds the low bits
    0101011."""
    S = np.array([3, 0, 2, 1, 3, 3, 0], np.uint8)
    b = np.unpackbits(O.wm_bits(S, 4), axis=1, bitorder="little")[:, :7]
    assert b[0].tolist() == [1, 0, 1, 0, 1, 1, 0]
    assert b[1].tolist() == [0, 1, 0, 1, 0, 1, 1]


def test_matrix_level_zero_and_sigma_two_equal_the_tree():
    """Level 0 of both is the top-bit plane of S, and with one level the two coincide."""
    S = inputs.zipf(4000, 96, 1.0, 3, np.uint8)
    assert np.array_equal(O.wm_bits(S, 96)[0], O.build_bits(S, 96)[0])
    T = inputs.uniform(4000, 2, 4, np.uint8)
    assert np.array_equal(O.wm_bits(T, 2), O.build_bits(T, 2))


@pytest.mark.parametrize("sigma", [2, 5, 20, 96, 256, 1000])
def test_matrix_ones_per_level_match_histogram(sigma):
    """Every level holds each symbol's bit once: ones_l = sum_c H[c] bit_l(c)."""
    S = inputs.zipf(5000, sigma, 1.1, 9, inputs.sym_dtype(sigma))
    L = O.levels(sigma)
    H = np.bincount(S, minlength=sigma)
    bits = O.wm_bits(S, sigma)
    for l in range(L):
        codes = np.arange(sigma)
        want = int((H * ((codes >> (L - 1 - l)) & 1)).sum())
        assert O.directory(bits[l], len(S))["ones"] == want


@pytest.mark.parametrize("sigma,n", [(2, 50), (5, 200), (17, 300), (64, 257), (256, 513), (1000, 700)])
def test_matrix_queries_against_brute_force(sigma, n):
    """access = S[i], rank = count of c in [0, i), select = position of the
    j-th c, all from S directly; sentinels for out-of-range arguments."""
    rng = np.random.default_rng(n + sigma)
    S = rng.integers(0, sigma, n).astype(inputs.sym_dtype(sigma))
    bits = O.wm_bits(S, sigma)
    I = np.arange(n + 2, dtype=np.uint64)
    acc = O.wm_access(bits, n, sigma, I)
    assert acc[:n].tolist() == S.tolist() and acc[n:].tolist() == [0xFFFFFFFF] * 2
    cs = rng.integers(0, sigma + 1, 400).astype(np.uint32)
    cs[: min(200, n)] = S[rng.integers(0, n, min(200, n))]
    ii = rng.integers(0, n + 2, 400).astype(np.uint64)
    want_r = [int((S[:i] == c).sum()) if (c < sigma and i <= n) else 2**64 - 1 for c, i in zip(cs, ii)]
    assert O.wm_rank(bits, n, sigma, cs, ii).tolist() == want_r
    jj = rng.integers(0, 12, 400).astype(np.uint64)
    want_s = []
    for c, j in zip(cs, jj):
        pos = np.flatnonzero(S == c) if c < sigma else []
        want_s.append(int(pos[j - 1]) if 1 <= j <= len(pos) else 2**64 - 1)
    assert O.wm_select(bits, n, sigma, cs, jj).tolist() == want_s


def test_matrix_sigma_one_has_no_levels():
    S = np.zeros(10, np.uint8)
    bits = O.wm_bits(S, 1)
    assert bits.shape == (0, 64)
    assert O.wm_access(bits, 10, 1, [0, 9, 10]).tolist() == [0, 0, 0xFFFFFFFF]
    assert O.wm_rank(bits, 10, 1, [0, 0], [4, 10]).tolist() == [4, 10]
    assert O.wm_select(bits, 10, 1, [0, 0], [1, 11]).tolist() == [0, 2**64 - 1]


# ------------------------------------------------------- alphabet remapping

@pytest.mark.parametrize("universe,alphabet,dtype", [
    (1 << 20, [0, 7, 1000, (1 << 20) - 1], np.uint32),
    (65536, [3, 4, 5, 60000, 65535], np.uint16),
    (256, [1, 2, 200, 255], np.uint8),
    (5, [4], np.uint8),
])
def test_remap_is_the_definition_and_queries_equal_brute_force(universe, alphabet, dtype):
    """Sparse alphabets: the bitmap marks exactly the codes that occur, S'
    is each code's rank among them, and access/rank/select through the
    remapped tree equal direct counting on S, for every argument."""
    rng = np.random.default_rng(len(alphabet) + universe)
    S = np.asarray(alphabet, dtype=dtype)[rng.integers(0, len(alphabet), 61)]
    bm, codes, Sr, sr = O.remap_alphabet(S, universe)
    present = np.unpackbits(bm, bitorder="little")
    assert present.shape[0] == ((universe + 511) // 512) * 512
    assert np.array_equal(np.flatnonzero(present), np.unique(S).astype(np.int64))
    assert list(codes) == sorted(set(int(x) for x in S))
    assert sr == len(codes)
    assert np.array_equal(Sr, np.array([list(codes).index(int(x)) for x in S], np.uint32))
    bits = O.build_bits(Sr, sr)
    n = len(S)
    I = np.arange(n + 2, dtype=np.uint64)
    want = [int(S[i]) if i < n else 0xFFFFFFFF for i in range(n + 2)]
    assert list(O.remap_access(codes, bits, n, sr, I)) == want
    absent = [c for c in range(min(universe, 1200)) if c not in set(alphabet)][:5]
    for c in list(alphabet) + absent + [universe, universe + 7]:
        cs = np.full(n + 2, c, np.uint64)
        r = O.remap_rank(codes, universe, bits, n, sr, cs, I)
        for i in range(n + 2):
            w = 2**64 - 1 if c >= universe or i > n else int(np.sum(S[:i] == c))
            assert int(r[i]) == w, (c, i)
        occ = np.flatnonzero(S == c) if c < universe else np.zeros(0, np.int64)
        J = np.arange(len(occ) + 2, dtype=np.uint64)
        got = O.remap_select(codes, universe, bits, n, sr, np.full(len(J), c, np.uint64), J)
        for j in range(len(J)):
            w = int(occ[j - 1]) if 1 <= j <= len(occ) else 2**64 - 1
            assert int(got[j]) == w, (c, j)


def test_remap_of_a_contiguous_alphabet_is_the_identity():
    S = inputs.uniform(5000, 96, 8, np.uint8)
    S[:96] = np.arange(96, dtype=np.uint8)   # every code occurs
    bm, codes, Sr, sr = O.remap_alphabet(S, 96)
    assert sr == 96 and np.array_equal(codes, np.arange(96)) and np.array_equal(Sr, S.astype(np.uint32))
    assert np.array_equal(O.build_bits(Sr, sr), O.build_bits(S, 96))


def test_remap_edge_cases():
    bm, codes, Sr, sr = O.remap_alphabet(np.zeros(0, np.uint8), 10)
    assert len(codes) == 0 and sr == 1 and len(Sr) == 0 and not bm.any()
    with pytest.raises(O.OracleError):
        O.remap_alphabet(np.array([3, 10], np.uint8), 10)
