"""Failure detection: a bounded device wait that runs out is reported as
WT_ERR_TIMEOUT and leaves the CUDA context usable.

The wait runs on an mbarrier that nothing completes (no copy targets it), for
a few milliseconds; nothing traps, faults or hangs."""
import numpy as np
import pytest

from gpu_helpers import compare_tree, needs_gpu, to_dev, wt
from paper_1610_05994_gb300 import inputs

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_wait_that_runs_out_is_a_timeout_and_the_context_survives():
    W = wt()
    assert W.wait_selftest(2_000_000, arrive=False) == W.ERR_TIMEOUT   # 2 ms, nothing arrives
    assert W.wait_selftest(2_000_000, arrive=True) == W.OK             # the same wait, completed
    assert W.wait_selftest(1_000, arrive=False) == W.ERR_TIMEOUT
    S = inputs.zipf(100_003, 96, 1.0, 3, np.uint8)
    compare_tree(W.Tree.build(to_dev(S), 96), S, 96)                    # the context still works


def test_wait_limit_is_checked_on_the_host():
    W = wt()
    assert W.wait_selftest(0, arrive=False) == W.ERR_ARG
    assert W.wait_selftest(2_000_000_000, arrive=False) == W.ERR_ARG
