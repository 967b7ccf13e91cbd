"""The locality stress inputs (Section 4, the cont and rand data sets): each
code of [0, sigma) appears n / sigma times, cont in code order, rand at the
positions of a seeded bijection; the numpy and torch generators agree."""
import numpy as np
import pytest

from paper_1610_05994_gb300 import inputs


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000, 4096, 5000, 1 << 16, 123457])
def test_positions_are_a_bijection(n):
    p = inputs.locality_positions(np.arange(n, dtype=np.uint64), n, 1234)
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint64))


@pytest.mark.parametrize("y", inputs.LOCALITY_SIZES)
def test_counts_and_order(y):
    sigma, n = 1 << y, 1 << 18
    cont = inputs.locality(n, sigma, "cont", 9)
    rand = inputs.locality(n, sigma, "rand", 9)
    assert np.all(np.bincount(cont, minlength=sigma) == n // sigma)
    assert np.all(np.diff(cont.astype(np.int64)) >= 0)
    assert np.array_equal(np.sort(rand), cont)
    # a random order: few positions keep their cont code
    assert np.mean(rand == cont) < 0.25


def test_ragged_length_counts_differ_by_at_most_one():
    a = inputs.locality(10007, 64, "rand", 3)
    c = np.bincount(a, minlength=64)
    assert c.max() - c.min() <= 1 and c.sum() == 10007


@pytest.mark.parametrize("n,sigma", [(1 << 12, 16), (5000, 64), (1 << 16, 1 << 14)])
@pytest.mark.parametrize("kind", ["cont", "rand"])
def test_numpy_and_torch_agree(n, sigma, kind):
    a = inputs.locality(n, sigma, kind, 21)
    b = inputs.locality_torch(n, sigma, kind, 21, "cpu").numpy().astype(np.uint32)
    assert np.array_equal(a, b)


def test_seeds_differ():
    assert not np.array_equal(inputs.locality(4096, 16, "rand", 1), inputs.locality(4096, 16, "rand", 2))
