"""The serving loop's host scheduling on CPU: admission by the device-memory
budget, eviction of the oldest resident trees, refusal of a request larger
than the whole budget, and a failed build giving back its bytes while the
rest of its batch retires.  Streams, events and the library's batched build
are replaced by fakes, so nothing here touches a GPU; the GPU tests run the
same loop on the real library."""
import contextlib

import pytest
import torch

from paper_1610_05994_gb300 import serve
from paper_1610_05994_gb300 import wt as W


class FakeStream:
    def __init__(self, device=None):
        self.waited_events = []

    def wait_stream(self, other):
        pass

    def wait_event(self, ev):
        self.waited_events.append(ev)


class FakeEvent:
    ready = True  # whether recorded work has finished (switched by the tests)

    def record(self, stream=None):
        pass

    def query(self):
        return FakeEvent.ready


class FakeSymbols:
    """Stands for a device tensor of n symbols of `width` bytes."""

    def __init__(self, n, width=1):
        self.n, self.width = n, width

    def numel(self):
        return self.n

    def element_size(self):
        return self.width

    def record_stream(self, stream):
        pass


class FakeTree:
    def __init__(self, fail):
        self.fail, self.freed = fail, False

    def wait(self):
        if self.fail:
            raise W.WTError(W.ERR_SYMBOL_RANGE, "wt_wait")

    def free(self):
        self.freed = True


@pytest.fixture
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: FakeStream())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: None)
    FakeEvent.ready = True
    calls = []

    def build_batch(seqs, sigmas, stream=None, wait=True):
        calls.append(len(seqs))
        return [FakeTree(getattr(S, "fail", False)) for S in seqs]

    monkeypatch.setattr(serve.W, "build_batch", build_batch)
    return calls


N, SIGMA = 1 << 20, 256
NEED = serve.tree_bytes(N, SIGMA, 1)   # bytes a build holds while it runs
KEEP = serve.resident_bytes(N, SIGMA)  # bytes its tree keeps


def _req(rid, n=N, fail=False):
    S = FakeSymbols(n)
    S.fail = fail
    return serve.BuildRequest(rid=rid, S=S, sigma=SIGMA, arrival=0.0)


def _server(budget, max_batch=1024):
    return serve.Server(budget_bytes=budget, max_batch=max_batch, device=torch.device("cpu"))


def test_budget_admits_what_fits_and_evicts_the_oldest(fake_cuda):
    srv = _server(NEED + KEEP - 1)
    r0, r1 = _req(0), _req(1)
    srv.submit(r0)
    srv.submit(r1)
    srv.step()  # r0 fits; r1 would exceed the budget and waits
    assert fake_cuda == [1] and srv.used == NEED and list(srv.queue) == [r1]
    srv.step()  # r0 retires (its scratch returns), then r1 needs r0 evicted
    assert r0.done > 0 and srv.evicted == 1 and srv.used == NEED
    assert fake_cuda == [1, 1] and not srv.queue
    srv.step()  # r1 retires
    assert list(srv.resident) == [1] and srv.used == KEEP
    assert srv.peak_used == NEED


def test_eviction_waits_for_the_queries_issued_before_it(fake_cuda):
    srv = _server(NEED + KEEP - 1)
    srv.submit(_req(0))
    srv.step()
    srv.step()  # r0 resident
    srv.last_query_event = FakeEvent()
    srv.submit(_req(1))
    srv.step()  # evicts r0: its free waits for the last query batch
    assert srv.evicted == 1 and srv.build_stream.waited_events == [srv.last_query_event]


def test_request_larger_than_the_budget_is_refused_without_evicting(fake_cuda):
    srv = _server(2 * NEED)
    srv.submit(_req(0))
    srv.step()
    srv.step()  # r0 resident
    big, small = _req(1, n=64 * N), _req(2)
    srv.submit(big)
    srv.submit(small)
    srv.step()
    assert srv.rejected == [big] and big.error and big.S is None
    assert srv.evicted == 0 and 0 in srv.resident  # nothing was evicted for it
    assert fake_cuda[-1] == 1 and not srv.queue    # the next request went on


def test_a_failed_build_gives_back_its_bytes_and_the_batch_retires(fake_cuda):
    srv = _server(10 * NEED)
    reqs = [_req(0), _req(1, fail=True), _req(2)]
    for r in reqs:
        srv.submit(r)
    srv.step()
    assert fake_cuda == [3] and srv.used == 3 * NEED
    FakeEvent.ready = False
    srv.step()  # still running: nothing retires
    assert srv.used == 3 * NEED and not srv.finished
    FakeEvent.ready = True
    srv.step()
    assert srv.failed == [reqs[1]] and reqs[1].error
    assert srv.finished == [reqs[0], reqs[2]]
    assert srv.used == 2 * KEEP and sorted(srv.resident) == [0, 2]
    assert srv.built_symbols == 2 * N


def test_batches_are_capped_and_keep_arrival_order(fake_cuda):
    srv = _server(10 * NEED, max_batch=2)
    reqs = [_req(k) for k in range(3)]
    for r in reqs:
        srv.submit(r)
    srv.step()
    srv.step()
    assert fake_cuda == [2, 1]
    srv.drain()
    assert [r.rid for r in srv.finished] == [0, 1, 2]
    srv.close()
    assert srv.used == 0 and not srv.resident
