"""GPU parity on the locality stress inputs (Section 4, cont and rand over
sigma = 2^y, y in {4, 6, ..., 14}, four-byte symbols): whole trees equal the
oracle's at sizes spanning many tiles, the device generator equals the host
one, and the benchmark's size (n = 2^30, y = 14, rand) passes the
size-independent checks."""
import numpy as np
import pytest
import torch

from gpu_helpers import compare_tree, needs_gpu, to_dev, wt
from test_gpu_fullsize import check_full
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.mark.parametrize("kind", ["cont", "rand"])
@pytest.mark.parametrize("y", inputs.LOCALITY_SIZES)
@pytest.mark.parametrize("n", [(1 << 16) + 1001, 1 << 17])
def test_locality_bit_exact(n, y, kind):
    W = wt()
    sigma = 1 << y
    S = inputs.locality(n, sigma, kind, 40 + y)
    t = W.Tree.build(to_dev(S), sigma)
    compare_tree(t, S, sigma)
    t.free()


@pytest.mark.parametrize("kind", ["cont", "rand"])
def test_device_generator_matches_host(kind):
    n, sigma = (1 << 20) + 77, 1 << 10
    a = inputs.locality(n, sigma, kind, 8)
    b = inputs.locality_torch(n, sigma, kind, 8, "cuda").cpu().numpy().astype(np.uint32)
    assert np.array_equal(a, b)


def test_full_size_rand():
    W = wt()
    n, sigma = 1 << 30, 1 << 14
    S = inputs.locality_torch(n, sigma, "rand", 1014, "cuda").cpu().numpy().astype(np.uint32)
    check_full(W, S, sigma, seed=14)
    del S
    torch.cuda.empty_cache()
