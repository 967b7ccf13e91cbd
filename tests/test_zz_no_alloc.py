"""The node-starts entry point that allocates no device memory.

Some callers of this library may not allocate device memory while they run
(a process that gives the whole device to its own pool at start-up, or a loop
that must not take the allocator's locks).  wt_node_starts_noalloc serves
them from a fixed scratch array compiled into the library.  Its answer must
equal the allocating wt_node_starts on the same input, call after call, even
though every call reuses (and must first clear) the same array.  This file
is collected last, so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from gpu_helpers import needs_gpu, to_dev, wt
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_noalloc_node_starts_match_allocating_entry_point_twice_in_a_row():
    W = wt()
    cases = [(inputs.zipf(1_000_003, 96, 1.0, 31, np.uint8), 96),
             (inputs.uniform(777_777, 65536, 32, np.uint16), 65536)]
    for S, sigma in cases:
        D = to_dev(S)
        want = W.node_starts(D, sigma).cpu().numpy()
        first = W.node_starts_noalloc(D, sigma).cpu().numpy()
        second = W.node_starts_noalloc(D, sigma).cpu().numpy()   # same array reused: cleared first
        assert np.array_equal(first, want)
        assert np.array_equal(second, want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    W = wt()
    D = to_dev(np.zeros(16, np.uint32))
    with pytest.raises(W.WTError) as e:
        W.node_starts_noalloc(D, (1 << 16) + 1)
    assert e.value.status == W.ERR_ARG
