"""Shared helpers of the GPU parity tests: build through the C ABI, read a tree
back, and compare it with the CPU oracle element by element."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1610_05994_gb300 import build as B
from paper_1610_05994_gb300 import inputs

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def wt():
    """The binding, with the library built (fast when up to date)."""
    from paper_1610_05994_gb300 import wt as W
    B.build_library()
    W.load()
    return W


def to_dev(S: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(S)).cuda()


def tree_bits(tree) -> np.ndarray:
    """(L, level_bytes) uint8 array of the tree's level bitmaps."""
    info = tree.info()
    L = info["levels"]
    lb = ((tree.n + 511) // 512) * 64
    out = np.zeros((L, lb), dtype=np.uint8)
    for l in range(L):
        out[l] = tree.level(l).words.cpu().numpy().view(np.uint8)
    return out


def compare_tree(tree, S: np.ndarray, sigma: int, check_dir: bool = True):
    """Bitmaps, directories and per-level ones of a GPU tree equal the oracle's."""
    want = O.build_bits(S, sigma)
    got = tree_bits(tree)
    assert got.shape == want.shape
    for l in range(want.shape[0]):
        if not np.array_equal(got[l], want[l]):
            bad = np.flatnonzero(got[l] != want[l])
            raise AssertionError(f"level {l}: {len(bad)} bytes differ, first at byte {bad[0]}")
        if check_dir:
            lv = tree.level(l)
            d = O.directory(want[l], len(S))
            assert np.array_equal(lv.R.cpu().numpy(), d["R"]), f"R level {l}"
            assert np.array_equal(lv.Hy.cpu().numpy(), d["Hy"]), f"Hy level {l}"
            assert np.array_equal(lv.S1.cpu().numpy(), d["S1"]), f"S1 level {l}"
            assert np.array_equal(lv.S0.cpu().numpy(), d["S0"]), f"S0 level {l}"
            assert lv.ones == d["ones"]
    return want


def query_batches(S: np.ndarray, sigma: int, m: int, seed: int):
    """Random plus edge queries: i in {0, n-1, n, n+1}, c in {0, sigma-1, sigma},
    j in {0, 1, count, count+1}."""
    rng = np.random.default_rng(seed)
    n = len(S)
    I = rng.integers(0, n + 2, m).astype(np.uint64)
    I[:4] = [0, max(n - 1, 0), n, n + 1]
    Cs = rng.integers(0, sigma + 1, m).astype(np.uint32)
    if n:
        pick = rng.integers(0, n, m // 2)
        Cs[: m // 2] = S[pick]
    Cs[:3] = [0, sigma - 1, sigma]
    counts = np.bincount(S, minlength=sigma + 1) if n else np.zeros(sigma + 1, np.int64)
    J = np.array([rng.integers(0, counts[c] + 2) for c in Cs], dtype=np.uint64)
    J[:4] = [0, 1, counts[Cs[2]], counts[Cs[3]] + 1]
    return I, Cs, J
