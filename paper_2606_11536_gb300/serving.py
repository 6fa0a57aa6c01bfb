"""Continuous-batching PIR serving over the C ABI.

Several NTT-encoded databases stay resident in HBM.  Requests (a database name and
one query: D1 ciphertexts) arrive over time into one FIFO queue per database.  The
server keeps `streams` CUDA streams as execution slots; whenever a slot is free it
takes the database whose oldest waiting request arrived first, coalesces up to that
database's batch cap of its waiting requests into one batch, gathers their queries
into the slot's batch buffer and issues the answer on the slot's stream.  Requests
that arrive while batches are running wait for the next free slot, so work from
different batches and databases overlaps on the device.

Limits and failure handling:
  - a batch is held back (or shrunk) until its device memory (query and response
    buffers and the answer's own scratch) fits the scratch budget left by the
    batches in flight;
  - a batch that cannot be started (the library or torch finds no memory for it,
    after the library's cached scratch has been given back) fails its requests
    with that status (PIR_ERR_OOM, 2) and the server goes on;
  - per database, a batch cap (`db_max_batch`) and a cap on the slots it may hold at
    once (`db_max_slots`), so that one large database cannot take every slot while
    the small ones wait behind its long batches;
  - a batch whose completion event has not fired `batch_timeout` seconds after its
    dispatch fails its requests with PIR_ERR_TIMEOUT (status 5, the C ABI's code);
    the slot keeps the batch's buffers and stays out of use until the event does
    fire, since the device may still write into them; once such a slot has waited
    another `batch_timeout`, requests that only stuck slots could take (their
    database's slot cap all stuck, or every slot stuck) fail with PIR_ERR_TIMEOUT
    too, instead of waiting behind batches that may never complete;
  - a request can be cancelled: a waiting one leaves its queue, a running one leaves
    its batch's results (the rest of the batch completes normally).
A database is admitted only if its resident bytes fit the memory budget (when one is
set) and the library's own free-HBM check (PIR_ERR_ADMISSION).

The scheduling logic is host code and runs against any backend with the small
interface below; `CudaBackend` is the real one (torch streams and events, the C
ABI, optionally captured graphs per database and batch size), tests also drive a
CPU fake.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import random
import time
from typing import Callable, Dict, List, Optional, Union

import numpy as np

from . import binding

PIR_OK = 0
PIR_ERR_OOM = 2
PIR_ERR_TIMEOUT = 5


@dataclasses.dataclass
class Request:
    rid: int
    db: str
    query: object            # backend query handle (a device tensor for CudaBackend)
    t_arrival: float
    t_dispatch: float = math.nan
    t_done: float = math.nan
    batch_size: int = 0
    response: object = None  # filled when keep_responses is set
    status: int = PIR_OK     # PIR_ERR_TIMEOUT when its batch ran out of time, PIR_ERR_OOM
                             # (or another status) when the batch could not be started
    cancelled: bool = False

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclasses.dataclass
class _Slot:
    stream: object
    busy: bool = False
    event: object = None
    requests: List[Request] = dataclasses.field(default_factory=list)
    db: str = ""
    bufs: object = None      # the batch's buffers, alive until the event completes
    scratch: int = 0
    t_dispatch: float = 0.0
    timed_out: bool = False  # requests already failed; the slot waits for its event


class Backend:
    """What the scheduler needs from the device side."""

    def setup_db(self, name, params, raw, layout):  # -> handle, resident bytes
        raise NotImplementedError

    def free_db(self, handle):
        raise NotImplementedError

    def new_stream(self):
        raise NotImplementedError

    def dispatch(self, handle, params, queries, stream):  # -> (event, buffers)
        raise NotImplementedError

    def done(self, event) -> bool:
        raise NotImplementedError

    def response(self, bufs, b: int, B: int):
        raise NotImplementedError

    def check(self) -> int:
        """Device-side status after a timeout (PIR_OK, or the library's error code)."""
        return PIR_OK


class AdmissionError(RuntimeError):
    pass


def _per_db(value, name, default):
    if value is None:
        return default
    if isinstance(value, dict):
        return value.get(name, default)
    return value


class Server:
    def __init__(self, backend: Backend, streams: int = 4, max_batch: int = 32, memory_budget: Optional[int] = None,
                 scratch_budget: Optional[int] = None, keep_responses: bool = False,
                 clock: Callable[[], float] = time.perf_counter, batch_timeout: Optional[float] = None,
                 db_max_batch: Union[None, int, Dict[str, int]] = None,
                 db_max_slots: Union[None, int, Dict[str, int]] = None):
        self.be = backend
        self.max_batch = max_batch
        self.budget = memory_budget
        self.scratch_budget = scratch_budget
        self.scratch_in_flight = 0
        self.keep = keep_responses
        self.clock = clock
        self.batch_timeout = batch_timeout
        self.db_max_batch = db_max_batch
        self.db_max_slots = db_max_slots
        self.dbs: Dict[str, dict] = {}
        self.queues: Dict[str, collections.deque] = {}
        self.slots = [_Slot(stream=backend.new_stream()) for _ in range(streams)]
        self.done: List[Request] = []       # answered requests
        self.failed: List[Request] = []     # requests whose batch timed out or could not start
        self.cancelled: List[Request] = []
        self.device_status = PIR_OK
        self.resident_bytes = 0

    # --- databases -----------------------------------------------------------
    def admit(self, name: str, params, raw, layout: int = 0) -> int:
        """Set up and keep database `name`; raises AdmissionError if it does not fit."""
        if name in self.dbs:
            raise ValueError("database %r already resident" % name)
        need = binding.resident_db_bytes(params, layout)
        if self.budget is not None and self.resident_bytes + need > self.budget:
            raise AdmissionError("%s needs %d bytes, %d of the %d-byte budget are left"
                                 % (name, need, self.budget - self.resident_bytes, self.budget))
        handle, nbytes = self.be.setup_db(name, params, raw, layout)
        self.dbs[name] = {"handle": handle, "params": params, "bytes": nbytes, "layout": layout}
        self.queues[name] = collections.deque()
        self.resident_bytes += nbytes
        return nbytes

    def evict(self, name: str):
        if self.queues[name] or any(s.busy and s.db == name for s in self.slots):
            raise RuntimeError("database %r still has work" % name)
        self.be.free_db(self.dbs[name]["handle"])
        self.resident_bytes -= self.dbs[name]["bytes"]
        del self.dbs[name], self.queues[name]

    # --- requests ------------------------------------------------------------
    def submit(self, req: Request):
        self.queues[req.db].append(req)

    def cancel(self, rid: int) -> bool:
        """Cancel request rid.  A waiting request leaves its queue at once; a running
        one is dropped from its batch's results when the batch completes.  Returns
        False if no waiting or running request has that id."""
        for q in self.queues.values():
            for r in q:
                if r.rid == rid:
                    q.remove(r)
                    r.cancelled = True
                    r.t_done = self.clock()
                    self.cancelled.append(r)
                    return True
        for s in self.slots:
            if s.busy and not s.timed_out:
                for r in s.requests:
                    if r.rid == rid and not r.cancelled:
                        r.cancelled = True
                        return True
        return False

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values()) + sum(
            len(s.requests) for s in self.slots if s.busy and not s.timed_out)

    def _retire(self, now) -> List[Request]:
        finished = []
        for s in self.slots:
            if not s.busy:
                continue
            if self.be.done(s.event):
                if s.timed_out:
                    # the overdue batch has completed at last: the device status (a
                    # bounded kernel wait that ran out?) can be read now without
                    # blocking on it
                    self.device_status = self.be.check()
                else:
                    for b, r in enumerate(s.requests):
                        r.t_done = now
                        if r.cancelled:
                            self.cancelled.append(r)
                            continue
                        if self.keep:
                            r.response = self.be.response(s.bufs, b, len(s.requests))
                        finished.append(r)
                self.scratch_in_flight -= s.scratch
                s.busy, s.requests, s.event, s.bufs, s.scratch, s.timed_out = False, [], None, None, 0, False
            elif self.batch_timeout is not None and not s.timed_out and now - s.t_dispatch > self.batch_timeout:
                # fail the requests now; the slot (and its buffers) stays held until
                # the event fires, since the device may still write into them
                s.timed_out = True
                for r in s.requests:
                    r.t_done = now
                    if r.cancelled:
                        self.cancelled.append(r)
                        continue
                    r.status = PIR_ERR_TIMEOUT
                    self.failed.append(r)
                # no device-status read here: it waits for the device's work, and the
                # overdue batch may never complete (the other slots go on meanwhile)
        return finished

    def _slots_of(self, name) -> int:
        return sum(1 for s in self.slots if s.busy and s.db == name)

    def _stuck(self, s, now) -> bool:
        # a batch that ran out of time, and then another batch_timeout without its
        # completion event firing: it may never end
        return s.busy and s.timed_out and now - s.t_dispatch > 2 * self.batch_timeout

    def _fail_behind_stuck_slots(self, now):
        """Waiting requests that no slot can ever take (every slot stuck, or every slot
        their database may hold stuck) fail with PIR_ERR_TIMEOUT instead of queueing
        behind batches that may never complete."""
        usable = sum(1 for s in self.slots if not self._stuck(s, now))
        for name, q in self.queues.items():
            if not q:
                continue
            cap = _per_db(self.db_max_slots, name, len(self.slots))
            stuck_held = sum(1 for s in self.slots if s.db == name and self._stuck(s, now))
            if usable == 0 or stuck_held >= cap:
                while q:
                    r = q.popleft()
                    r.t_done = now
                    r.status = PIR_ERR_TIMEOUT
                    self.failed.append(r)

    def poll(self) -> List[Request]:
        """Retire finished batches (and time out overdue ones), then fill every free
        slot.  Returns the requests answered in this call."""
        now = self.clock()
        finished = self._retire(now)
        if self.batch_timeout is not None:
            self._fail_behind_stuck_slots(now)
        for s in self.slots:
            if s.busy:
                continue
            name = self._next_db()
            if name is None:
                break
            q = self.queues[name]
            info = self.dbs[name]
            p = info["params"]
            # one request's device memory while its batch runs: its query and response
            # buffers and the answer's own scratch (NTT-form copy, GEMM layout, result)
            per_query = 8 * p.L * p.n * (p.D1 + p.D2) + binding.answer_scratch_bytes(p, info.get("layout", 0), 1)
            nb = min(self.max_batch, _per_db(self.db_max_batch, name, self.max_batch), len(q))
            if self.scratch_budget is not None:
                nb = min(nb, (self.scratch_budget - self.scratch_in_flight) // per_query)
                if nb <= 0:
                    if self.scratch_in_flight:
                        break  # wait for batches in flight to release memory
                    nb = 1  # a single request larger than the budget still runs, alone
            take = [q.popleft() for _ in range(nb)]
            t = self.clock()
            for r in take:
                r.t_dispatch, r.batch_size = t, len(take)
            try:
                s.event, s.bufs = self.be.dispatch(info["handle"], p, [r.query for r in take], s.stream)
            except binding.PirError as e:
                # the batch could not be started (no memory for it): its requests fail
                # with the library's status and the slot stays free
                for r in take:
                    r.t_done = self.clock()
                    r.status = e.status
                    self.failed.append(r)
                continue
            s.busy, s.requests, s.db, s.scratch, s.t_dispatch = True, take, name, nb * per_query, t
            self.scratch_in_flight += s.scratch
        self.done.extend(finished)
        return finished

    def _next_db(self) -> Optional[str]:
        """The database whose oldest waiting request arrived first, among those
        below their slot cap."""
        best, t_best = None, math.inf
        for name, q in self.queues.items():
            if not q or q[0].t_arrival >= t_best:
                continue
            cap = _per_db(self.db_max_slots, name, len(self.slots))
            if self._slots_of(name) >= cap:
                continue
            best, t_best = name, q[0].t_arrival
        return best

    # --- open-loop run ---------------------------------------------------------
    def run(self, arrivals: List[Request], idle_sleep: float = 20e-6) -> List[Request]:
        """Serve requests whose t_arrival are offsets (s) from the start; returns them
        with t_arrival / t_dispatch / t_done on the server clock."""
        t0 = self.clock()
        todo = sorted(arrivals, key=lambda r: r.t_arrival)
        for r in todo:
            r.t_arrival += t0
        i = 0
        while i < len(todo) or self.pending():
            now = self.clock()
            while i < len(todo) and todo[i].t_arrival <= now:
                self.submit(todo[i])
                i += 1
            finished = self.poll()
            if not finished and i < len(todo) and not self.pending():
                wait = todo[i].t_arrival - self.clock()
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
            elif not finished:
                time.sleep(idle_sleep)
        return todo


def poisson_arrivals(rate_qps: float, duration_s: float, dbs: List[str], seed: int,
                     make_query: Callable[[str, int], object]) -> List[Request]:
    """Open-loop Poisson arrivals at rate_qps for duration_s, each to a uniformly
    random database; make_query(db, k) supplies the query handle."""
    rng = random.Random(seed)
    t, k, out = 0.0, 0, []
    while True:
        t += rng.expovariate(rate_qps)
        if t >= duration_s:
            return out
        db = dbs[rng.randrange(len(dbs))]
        out.append(Request(rid=k, db=db, query=make_query(db, k), t_arrival=t))
        k += 1


def latency_stats(reqs: List[Request]) -> dict:
    ok = [r for r in reqs if not math.isnan(r.t_done) and r.status == PIR_OK and not r.cancelled]
    lat = np.array([r.latency for r in ok]) * 1e3
    if lat.size == 0:
        return {"count": 0}
    span = max(r.t_done for r in ok) - min(r.t_arrival for r in ok)
    return {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "qps": float(lat.size / span) if span > 0 else 0.0,
            "mean_batch": float(np.mean([r.batch_size for r in ok])),
            "failed": sum(1 for r in reqs if r.status != PIR_OK),
            "cancelled": sum(1 for r in reqs if r.cancelled)}


def graph_bucket(B: int, max_batch: int) -> int:
    """Batch size a captured graph is made for: the next power of two (at most
    max_batch), so a few graphs per database serve every batch size."""
    b = 1
    while b < B:
        b <<= 1
    return max(B, min(b, max_batch))


class CudaBackend(Backend):
    """The real backend: the C ABI for the scan, torch for buffers, streams and events.

    Without graphs, every dispatch allocates its batch buffers through torch and
    calls pir_answer; with large databases run the process with torch's
    stream-ordered allocator (PYTORCH_CUDA_ALLOC_CONF=backend:cudaMallocAsync), whose
    releases do not synchronise the device as the caching allocator's do under
    memory pressure.

    With graphs=True, a batch runs as one captured answer (pir_graph_create) per
    (database, batch bucket, slot): the batch is padded with zero queries to the
    bucket (graph_bucket), whose tile and K-chunk the library's autotuner picks once
    per (database, bucket).  The graph's query and response buffers stay bound to it;
    a slot runs one batch at a time, so its graphs' buffers are free whenever the
    slot is.  Graphs are kept within graph_budget bytes of bound buffers, least
    recently used first out; a graph above an eighth of the budget is not made, and
    such a batch, like any that does not fit, runs uncaptured.  prewarm() makes the
    graphs before serving starts."""

    def __init__(self, device: int = 0, graphs: bool = False, max_batch: int = 32, graph_budget: int = 16 << 30,
                 autotune: bool = True):
        import torch

        import paper_2606_11536_gb300 as g
        self.torch, self.g = torch, g
        self.device = torch.device("cuda", device)
        self.graphs = graphs
        self.max_batch = max_batch
        self.graph_budget = graph_budget
        self.autotune = autotune
        self._graphs = collections.OrderedDict()  # (db id, bucket, stream id) -> [graph, qbuf, rbuf, bytes, event]
        self._graph_bytes = 0
        self._tuned: Dict[tuple, dict] = {}
        self.graph_launches = 0
        self.frozen = False  # set by prewarm(): no graph is made while serving

    def setup_db(self, name, params, raw, layout):
        try:
            db = self.g.pir_setup_db(params, raw, layout=layout)
        except self.g.PirError as e:
            if e.status == 3:
                raise AdmissionError("%s: %s" % (name, e)) from e
            raise
        return db, self.g.pir_db_bytes(db)

    def free_db(self, handle):
        self.torch.cuda.synchronize(self.device)
        for key in [k for k in self._graphs if k[0] == id(handle)]:
            self._drop_graph(key)
        self.g.pir_free_db(handle)

    def new_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def _empty(self, words):
        """A batch buffer from torch; if torch finds no room, the memory the library
        keeps cached (answer and graph scratch) is given back and the allocation
        tried once more."""
        torch = self.torch
        try:
            return torch.empty(words, dtype=torch.int32, device=self.device)
        except torch.OutOfMemoryError:
            self.g.pir_release_memory()
        try:
            return torch.empty(words, dtype=torch.int32, device=self.device)
        except torch.OutOfMemoryError as e:
            raise self.g.PirError(PIR_ERR_OOM, "batch buffer", str(e)) from e

    def _drop_graph(self, key):
        graph, _, _, nbytes, _ = self._graphs.pop(key)
        self.g.pir_graph_destroy(graph)
        self._graph_bytes -= nbytes

    def prewarm(self, server, buckets=None):
        """Autotune and capture the graphs of every resident database, batch bucket
        and slot ahead of serving (a server does this at start-up, so the first
        requests do not pay for it).  Skips what does not fit the graph budget."""
        buckets = buckets or sorted({graph_bucket(b, self.max_batch) for b in range(1, self.max_batch + 1)})
        for name, info in server.dbs.items():
            for bucket in buckets:
                for slot in server.slots:
                    self._graph_for(info["handle"], info["params"], bucket, slot.stream)
        self.torch.cuda.synchronize(self.device)
        # from here on no graph is made while serving (a capture synchronizes the
        # device): a batch without a graph runs uncaptured
        self.frozen = True

    def _graph_for(self, handle, params, bucket, stream):
        key = (id(handle), bucket, id(stream))
        if key in self._graphs:
            self._graphs.move_to_end(key)
            return self._graphs[key]
        if self.frozen:
            return None
        torch = self.torch
        qwords = bucket * params.D1 * 2 * params.L * params.n
        rwords = bucket * params.D2 * 2 * params.L * params.n
        nbytes = 4 * (qwords + rwords)
        if nbytes > self.graph_budget // 8:
            # a graph this large would crowd out the others: such batches run uncaptured,
            # rather than evicting and re-capturing graphs batch after batch
            return None
        while self._graph_bytes + nbytes > self.graph_budget:
            # least recently used first, and never a graph whose last launch is still
            # running (its bound buffers are in use)
            idle = next((k for k, e in self._graphs.items() if e[4] is None or e[4].query()), None)
            if idle is None:
                return None
            self._drop_graph(idle)
        tkey = (id(handle), bucket)
        if tkey not in self._tuned:
            self._tuned[tkey] = self.g.pir_autotune(handle, bucket, stream=stream) if self.autotune else \
                {"tile": 0, "k_chunk": 0}
        opts = self._tuned[tkey]
        qbuf = torch.zeros(qwords, dtype=torch.int32, device=self.device)
        rbuf = torch.empty(rwords, dtype=torch.int32, device=self.device)
        torch.cuda.synchronize(self.device)  # buffers written before the capture reads them
        graph = self.g.pir_graph_create(handle, qbuf, bucket, rbuf, k_chunk=opts["k_chunk"], tile=opts["tile"])
        entry = [graph, qbuf, rbuf, nbytes, None]  # last: the event of its latest launch
        self._graphs[key] = entry
        self._graph_bytes += nbytes
        return entry

    def dispatch(self, handle, params, queries, stream):
        torch = self.torch
        B = len(queries)
        qwords = params.D1 * 2 * params.L * params.n
        rwords = params.D2 * 2 * params.L * params.n
        entry = None
        if self.graphs:
            entry = self._graph_for(handle, params, graph_bucket(B, self.max_batch), stream)
        with torch.cuda.stream(stream):
            if entry is not None:
                graph, qbuf, rbuf = entry[0], entry[1], entry[2]
                for b, q in enumerate(queries):  # gather into the graph's bound buffer
                    qbuf[b * qwords:(b + 1) * qwords].copy_(q, non_blocking=True)
                if B * qwords < qbuf.numel():
                    qbuf[B * qwords:].zero_()  # padding rows: zero queries, answers discarded
                self.g.pir_graph_launch(graph, stream=stream)
                self.graph_launches += 1
                bufs = (qbuf, rbuf[:B * rwords])
            else:
                qbuf = self._empty(B * qwords)
                for b, q in enumerate(queries):  # gather: one device-to-device copy per request
                    qbuf[b * qwords:(b + 1) * qwords].copy_(q, non_blocking=True)
                rbuf = self._empty(B * rwords)
                self.g.pir_answer(handle, qbuf, B, rbuf, stream=stream)
                bufs = (qbuf, rbuf)
            ev = torch.cuda.Event()
            ev.record(stream)
        if entry is not None:
            entry[4] = ev
        return ev, bufs

    def done(self, event) -> bool:
        return event.query()

    def check(self) -> int:
        try:
            self.g.pir_device_status()  # waits for no work: other slots may still run
        except self.g.PirError as e:
            return e.status
        return PIR_OK

    def response(self, bufs, b: int, B: int):
        rbuf = bufs[1]
        per = rbuf.numel() // B
        return rbuf[b * per:(b + 1) * per].clone()
