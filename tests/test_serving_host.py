"""Host-side serving logic (continuous batching, admission) against a CPU fake of
the device backend: no GPU involved."""
import types

import pytest

from paper_2606_11536_gb300.serving import AdmissionError, Backend, Request, Server, latency_stats, poisson_arrivals


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend(Backend):
    """A batch finishes `latency` fake seconds after dispatch; the 'answer' of a
    query q against database d is (d.salt, q)."""

    def __init__(self, clock, latency=1.0):
        self.clock, self.latency = clock, latency
        self.batches = []

    def setup_db(self, name, params, raw, layout):
        return types.SimpleNamespace(name=name, salt=hash(name) % 1000), 4 * params.L * params.n * params.D1 * params.D2

    def free_db(self, handle):
        pass

    def new_stream(self):
        return object()

    def dispatch(self, handle, params, queries, stream):
        self.batches.append((handle.name, list(queries)))
        return self.clock() + self.latency, [(handle.salt, q) for q in queries]

    def done(self, event):
        return self.clock() >= event

    def response(self, bufs, b, B):
        assert len(bufs) == B
        return bufs[b]


def params(n=2048, D1=16, D2=16):
    return types.SimpleNamespace(n=n, L=2, D1=D1, D2=D2, log2p=16)


def make(streams=2, max_batch=4, **kw):
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, streams=streams, max_batch=max_batch, clock=clock, keep_responses=True, **kw)
    return clock, be, srv


def test_requests_arriving_during_a_batch_are_coalesced():
    clock, be, srv = make(streams=1, max_batch=4)
    srv.admit("a", params(), None)
    srv.submit(Request(0, "a", 0, 0.0))
    srv.poll()                       # request 0 goes out alone
    for k in range(1, 7):            # six arrive while it runs
        srv.submit(Request(k, "a", k, 0.1 * k))
    srv.poll()
    assert [len(q) for _, q in be.batches] == [1]
    clock.t = 1.0
    srv.poll()                       # slot frees: next batch takes 4 (max_batch)
    assert [len(q) for _, q in be.batches] == [1, 4]
    clock.t = 2.0
    srv.poll()
    assert [len(q) for _, q in be.batches] == [1, 4, 2]
    clock.t = 3.0
    srv.poll()
    assert srv.pending() == 0 and len(srv.done) == 7
    assert [r.rid for r in srv.done] == list(range(7))  # FIFO within a database


def test_oldest_waiting_request_picks_the_database_and_slots_overlap():
    clock, be, srv = make(streams=2, max_batch=8)
    for name in ("a", "b", "c"):
        srv.admit(name, params(), None)
    srv.submit(Request(0, "b", 0, 0.0))
    srv.submit(Request(1, "a", 1, 0.1))
    srv.submit(Request(2, "c", 2, 0.2))
    srv.submit(Request(3, "b", 3, 0.3))
    srv.poll()
    # two slots: b (oldest head, takes both of its requests) and then a
    assert [name for name, _ in be.batches] == ["b", "a"]
    assert be.batches[0][1] == [0, 3]
    clock.t = 1.0
    srv.poll()
    assert [name for name, _ in be.batches] == ["b", "a", "c"]
    clock.t = 2.0
    srv.poll()
    assert srv.pending() == 0
    for r in srv.done:  # every response is the one its own query gives alone
        assert r.response == (hash(r.db) % 1000, r.query)


def test_admission_by_memory_budget():
    p = params(n=4096, D1=512, D2=256)  # 4 GiB resident
    clock, be, srv = make(memory_budget=9 << 30)
    srv.admit("a", p, None)
    srv.admit("b", p, None)
    with pytest.raises(AdmissionError):
        srv.admit("c", p, None)
    srv.evict("b")
    srv.admit("c", p, None)
    assert srv.resident_bytes == 8 << 30


def test_layout_reaches_the_backend_and_admission_counts_its_bytes():
    """The layout given to admit reaches the backend, and the budget check counts the
    tensor layout's 8 bytes per residue (twice the plain layout's)."""
    p = params(n=4096, D1=512, D2=256)  # 4 GiB resident plain, 8 GiB in the tensor layout
    clock, be, srv = make(memory_budget=10 << 30)
    seen = []
    setup = be.setup_db

    def recording_setup(name, params_, raw, layout):
        seen.append(layout)
        h, nbytes = setup(name, params_, raw, layout)
        return h, nbytes * (2 if layout == 2 else 1)

    be.setup_db = recording_setup
    srv.admit("plain", p, None)
    with pytest.raises(AdmissionError):  # 4 + 8 GiB exceed the 10 GiB budget
        srv.admit("tensor", p, None, layout=2)
    srv.admit("limb", p, None, layout=1)  # 4 + 4 GiB fit
    assert seen == [0, 1]
    assert srv.resident_bytes == 8 << 30


def test_scratch_budget_limits_batches_in_flight():
    from paper_2606_11536_gb300 import binding
    p = params(n=2048, D1=16, D2=16)
    # buffers (query + response) and the library's own scratch for one query
    per_query = 8 * 2 * 2048 * 32 + binding.answer_scratch_bytes(p, 0, 1)
    clock, be, srv = make(streams=3, max_batch=8, scratch_budget=5 * per_query)
    srv.admit("a", p, None)
    for k in range(12):
        srv.submit(Request(k, "a", k, 0.0))
    srv.poll()
    # first slot takes 5 (budget), the others wait for memory
    assert [len(q) for _, q in be.batches] == [5]
    clock.t = 1.0
    srv.poll()
    assert [len(q) for _, q in be.batches] == [5, 5]
    clock.t = 2.0
    srv.poll()
    clock.t = 3.0
    srv.poll()
    assert srv.pending() == 0 and sum(len(q) for _, q in be.batches) == 12


def test_open_loop_run_and_stats():
    import time as _time
    be_clock = _time.perf_counter
    calls = []

    class RealTimeFake(FakeBackend):
        def dispatch(self, handle, params, queries, stream):
            calls.append(len(queries))
            return be_clock() + 0.002, list(queries)

        def done(self, event):
            return be_clock() >= event

    srv = Server(RealTimeFake(be_clock), streams=2, max_batch=4)
    for name in ("a", "b"):
        srv.admit(name, params(), None)
    arr = poisson_arrivals(2000.0, 0.05, ["a", "b"], seed=3, make_query=lambda db, k: k)
    out = srv.run(arr)
    st = latency_stats(out)
    assert st["count"] == len(arr) > 40
    assert 2.0 <= st["p50_ms"] <= st["p99_ms"] < 200
    assert max(calls) <= 4 and sum(calls) == len(arr)


class StuckBackend(FakeBackend):
    """A fake whose batches complete only when the test says so, and whose device
    check reports a bounded wait that ran out."""

    def __init__(self, clock):
        super().__init__(clock)
        self.released = set()
        self.checks = 0

    def dispatch(self, handle, params, queries, stream):
        self.batches.append((handle.name, list(queries)))
        return len(self.batches) - 1, [(handle.salt, q) for q in queries]

    def done(self, event):
        return event in self.released

    def check(self):
        self.checks += 1
        return 5


def test_batch_timeout_fails_its_requests_and_holds_the_slot():
    clock = FakeClock()
    be = StuckBackend(clock)
    srv = Server(be, streams=1, max_batch=4, clock=clock, keep_responses=True, batch_timeout=2.0)
    srv.admit("a", params(), None)
    for k in range(2):
        srv.submit(Request(k, "a", k, 0.0))
    srv.poll()
    clock.t = 1.0
    assert srv.poll() == [] and not srv.failed
    clock.t = 2.5
    srv.submit(Request(2, "a", 2, 2.5))
    assert srv.poll() == []
    assert [r.rid for r in srv.failed] == [0, 1] and all(r.status == 5 for r in srv.failed)
    # no device-status read yet: it would wait for the overdue batch, which may never end
    assert srv.device_status == 0 and be.checks == 0
    assert len(be.batches) == 1          # the held slot takes no new batch
    assert srv.pending() == 1            # only the waiting request counts
    clock.t = 3.0
    be.released.add(0)                   # the stuck batch's event finally fires
    srv.poll()
    assert srv.device_status == 5 and be.checks == 1  # read once the batch has ended
    assert len(be.batches) == 2 and be.batches[1][1] == [2]
    assert srv.done == []                # the failed requests are not reported twice
    be.released.add(1)
    clock.t = 3.5
    srv.poll()
    assert [r.rid for r in srv.done] == [2] and srv.done[0].response[1] == 2
    stats = latency_stats([r for r in srv.failed] + srv.done)
    assert stats["count"] == 1 and stats["failed"] == 2


def test_cancel_a_waiting_and_a_running_request():
    clock, be, srv = make(streams=1, max_batch=2)
    srv.admit("a", params(), None)
    for k in range(4):
        srv.submit(Request(k, "a", k, 0.0))
    srv.poll()                           # 0 and 1 running, 2 and 3 waiting
    assert srv.cancel(3) and srv.cancel(1)
    assert not srv.cancel(99)
    clock.t = 1.0
    srv.poll()                           # batch {0, 1} completes; 2 goes out alone
    assert [r.rid for r in srv.done] == [0] and srv.done[0].response[1] == 0
    assert sorted(r.rid for r in srv.cancelled) == [1, 3]
    assert be.batches[1][1] == [2]
    clock.t = 2.0
    srv.poll()
    assert [r.rid for r in srv.done] == [0, 2] and srv.pending() == 0
    assert all(r.response is None for r in srv.cancelled)


def test_per_database_batch_and_slot_caps():
    clock, be, srv = make(streams=3, max_batch=8, db_max_batch={"big": 2}, db_max_slots={"big": 1})
    srv.admit("big", params(D1=64), None)
    srv.admit("small", params(), None)
    for k in range(6):
        srv.submit(Request(k, "big", k, 0.0))
    srv.submit(Request(10, "small", 10, 0.1))
    srv.poll()
    # big holds one slot with a batch of 2; small takes another slot at once
    assert [(d, len(q)) for d, q in be.batches] == [("big", 2), ("small", 1)]
    clock.t = 1.0
    srv.poll()
    assert [(d, len(q)) for d, q in be.batches][2:] == [("big", 2)]
    clock.t = 2.0
    srv.poll()
    clock.t = 3.0
    srv.poll()
    assert srv.pending() == 0 and len(srv.done) == 7


def test_answer_scratch_bytes_per_layout():
    from paper_2606_11536_gb300 import binding
    p = params(n=4096, D1=4096, D2=512)
    ct = 2 * 2 * 4096 * 4  # one ciphertext: 2 polynomials x L primes x n residues x 4 bytes
    # NTT-form copy + GEMM layout (4 bytes per residue; bf16 digits: 8) + result
    assert binding.answer_scratch_bytes(p, binding.PIR_LAYOUT_PLAIN, 1) == 2 * 4096 * ct + 512 * ct
    assert binding.answer_scratch_bytes(p, binding.PIR_LAYOUT_TENSOR, 1) == 3 * 4096 * ct + 512 * ct
    assert binding.answer_scratch_bytes(p, binding.PIR_LAYOUT_TENSOR, 32) == 32 * (3 * 4096 + 512) * ct


def test_a_batch_that_cannot_start_fails_its_requests_and_the_server_goes_on():
    from paper_2606_11536_gb300 import binding

    class FlakyBackend(FakeBackend):
        def __init__(self, clock):
            super().__init__(clock)
            self.refuse = 1  # the first dispatch finds no memory

        def dispatch(self, handle, params, queries, stream):
            if self.refuse:
                self.refuse -= 1
                raise binding.PirError(2, "batch buffer")
            return super().dispatch(handle, params, queries, stream)

    clock = FakeClock()
    be = FlakyBackend(clock)
    srv = Server(be, streams=1, max_batch=4, clock=clock, keep_responses=True)
    srv.admit("a", params(), None)
    for k in range(6):
        srv.submit(Request(k, "a", k, 0.0))
    srv.poll()  # the first 4 are refused; the slot stays free
    assert [r.rid for r in srv.failed] == [0, 1, 2, 3] and all(r.status == 2 for r in srv.failed)
    assert be.batches == [] and srv.pending() == 2
    srv.poll()  # the next poll gives it the remaining 2
    assert [q for _, q in be.batches] == [[4, 5]]
    clock.t = 1.0
    srv.poll()
    assert sorted(r.rid for r in srv.done) == [4, 5] and srv.pending() == 0


def test_requests_behind_stuck_slots_fail_instead_of_waiting_forever():
    clock = FakeClock()
    be = StuckBackend(clock)
    srv = Server(be, streams=2, max_batch=2, clock=clock, keep_responses=True, batch_timeout=2.0,
                 db_max_slots={"a": 1})
    srv.admit("a", params(), None)
    srv.admit("b", params(), None)
    srv.submit(Request(0, "a", 0, 0.0))
    srv.poll()                               # a's batch never completes
    srv.submit(Request(1, "a", 1, 0.5))
    clock.t = 2.5
    srv.poll()                               # it runs out of time: request 0 fails
    assert [r.rid for r in srv.failed] == [0]
    assert srv.pending() == 1                # request 1 still waits: the slot may yet free
    clock.t = 4.5                            # another timeout later the slot counts as stuck
    srv.submit(Request(2, "b", 2, 4.5))
    srv.poll()
    assert [r.rid for r in srv.failed] == [0, 1] and srv.failed[1].status == 5
    assert [q for _, q in be.batches] == [[0], [2]]  # database b still runs on the other slot
    be.released.add(1)
    clock.t = 5.0
    srv.poll()
    assert [r.rid for r in srv.done] == [2] and srv.pending() == 0
