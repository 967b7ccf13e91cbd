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


def test_noalloc_refuses_a_misaligned_input_on_the_host():
    """Two-byte symbols at an odd address: WT_ERR_ARG before any launch, and
    the next call still works (no sticky CUDA error)."""
    import ctypes as C

    import torch
    W = wt()
    S = inputs.uniform(10_001, 1000, 33, np.uint16)
    raw = torch.zeros(2 * len(S) + 2, dtype=torch.uint8, device="cuda")
    raw[1:1 + 2 * len(S)] = torch.from_numpy(S.view(np.uint8)).cuda()
    hex_ = torch.empty((1 << 10) + 1, dtype=torch.uint64, device="cuda")
    st = W.load().wt_node_starts_noalloc(C.c_void_p(raw.data_ptr() + 1), len(S), 1000, 2,
                                         C.c_void_p(hex_.data_ptr()), None)
    assert st == W.ERR_ARG
    D = to_dev(S)
    assert np.array_equal(W.node_starts_noalloc(D, 1000).cpu().numpy(), W.node_starts(D, 1000).cpu().numpy())


def test_noalloc_checks_the_output_tensor():
    import torch
    W = wt()
    D = to_dev(inputs.uniform(1000, 96, 3, np.uint8))
    for bad in (torch.empty(100, dtype=torch.uint64, device="cuda"),      # 2^7 + 1 needed
                torch.empty(129, dtype=torch.int32, device="cuda"),
                torch.empty(129, dtype=torch.uint64)):                    # host memory
        with pytest.raises(ValueError):
            W.node_starts_noalloc(D, 96, out=bad)


def test_noalloc_error_word_is_cleared_between_calls():
    """A call that finds a symbol >= sigma reports it; the next valid call on
    the same array returns the allocating entry point's answer."""
    W = wt()
    S = inputs.uniform(300_001, 200, 34, np.uint8)
    bad = S.copy()
    bad[123_456] = 250
    with pytest.raises(W.WTError) as e:
        W.node_starts_noalloc(to_dev(bad), 200)
    assert e.value.status == W.ERR_SYMBOL_RANGE
    D = to_dev(S)
    assert np.array_equal(W.node_starts_noalloc(D, 200).cpu().numpy(), W.node_starts(D, 200).cpu().numpy())


def test_noalloc_call_allocates_no_device_memory():
    """Neither PyTorch's allocator nor the device's free memory moves across
    a warm call (its scratch is the library's fixed array)."""
    import torch
    W = wt()
    D = to_dev(inputs.zipf(2_000_003, 4096, 1.1, 35, np.uint16))
    out = torch.empty((1 << 12) + 1, dtype=torch.uint64, device="cuda")
    W.node_starts_noalloc(D, 4096, out=out)   # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        W.node_starts_noalloc(D, 4096, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(out.cpu().numpy(), W.node_starts(D, 4096).cpu().numpy())
