"""Continuous-batching PIR serving over the C ABI.

Several NTT-encoded databases stay resident in HBM.  Requests (a database name and
one query: D1 ciphertexts) arrive over time into one FIFO queue per database.  The
server keeps `streams` CUDA streams as execution slots; whenever a slot is free it
takes the database whose oldest waiting request arrived first, coalesces up to
`max_batch` of that database's waiting requests into one batch, gathers their
queries into the slot's batch buffer and issues pir_answer on the slot's stream.
Requests that arrive while batches are running wait for the next free slot, so
work from different batches and databases overlaps on the device.  A batch is
also held back (or shrunk) until its query and response buffers fit the scratch
budget left by the batches in flight.  A database is admitted only if its resident
bytes fit the memory budget (when one is set) and the library's own free-HBM
check (PIR_ERR_ADMISSION).

The scheduling logic is host code and runs against any backend with the small
interface below; `CudaBackend` is the real one (torch streams and events, the C
ABI), tests also drive a CPU fake.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import random
import time
from typing import Callable, Dict, List, Optional

import numpy as np


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


class AdmissionError(RuntimeError):
    pass


class Server:
    def __init__(self, backend: Backend, streams: int = 4, max_batch: int = 32, memory_budget: Optional[int] = None,
                 scratch_budget: Optional[int] = None, keep_responses: bool = False,
                 clock: Callable[[], float] = time.perf_counter):
        self.be = backend
        self.max_batch = max_batch
        self.budget = memory_budget
        self.scratch_budget = scratch_budget
        self.scratch_in_flight = 0
        self.keep = keep_responses
        self.clock = clock
        self.dbs: Dict[str, dict] = {}
        self.queues: Dict[str, collections.deque] = {}
        self.slots = [_Slot(stream=backend.new_stream()) for _ in range(streams)]
        self.done: List[Request] = []
        self.resident_bytes = 0

    # --- databases -----------------------------------------------------------
    def admit(self, name: str, params, raw, layout: int = 0) -> int:
        """Set up and keep database `name`; raises AdmissionError if it does not fit."""
        if name in self.dbs:
            raise ValueError("database %r already resident" % name)
        # resident bytes per residue: u32 words or four u8 limbs (plain, limb), four
        # bf16 digits (the tensor layout, 2)
        need = (8 if layout == 2 else 4) * params.L * params.n * params.D1 * params.D2
        if self.budget is not None and self.resident_bytes + need > self.budget:
            raise AdmissionError("%s needs %d bytes, %d of the %d-byte budget are left"
                                 % (name, need, self.budget - self.resident_bytes, self.budget))
        handle, nbytes = self.be.setup_db(name, params, raw, layout)
        self.dbs[name] = {"handle": handle, "params": params, "bytes": nbytes}
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

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values()) + sum(len(s.requests) for s in self.slots if s.busy)

    def poll(self) -> List[Request]:
        """Retire finished batches, then fill every free slot.  Returns the requests
        that finished in this call."""
        finished = []
        now = self.clock()
        for s in self.slots:
            if s.busy and self.be.done(s.event):
                for b, r in enumerate(s.requests):
                    r.t_done = now
                    if self.keep:
                        r.response = self.be.response(s.bufs, b, len(s.requests))
                finished.extend(s.requests)
                self.scratch_in_flight -= s.scratch
                s.busy, s.requests, s.event, s.bufs, s.scratch = False, [], None, None, 0
        for s in self.slots:
            if s.busy:
                continue
            name = self._next_db()
            if name is None:
                break
            q = self.queues[name]
            info = self.dbs[name]
            p = info["params"]
            per_query = 8 * p.L * p.n * (p.D1 + p.D2)  # query + response words of one request
            nb = min(self.max_batch, len(q))
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
            s.event, s.bufs = self.be.dispatch(info["handle"], p, [r.query for r in take], s.stream)
            s.busy, s.requests, s.db, s.scratch = True, take, name, nb * per_query
            self.scratch_in_flight += s.scratch
        self.done.extend(finished)
        return finished

    def _next_db(self) -> Optional[str]:
        best, t_best = None, math.inf
        for name, q in self.queues.items():
            if q and q[0].t_arrival < t_best:
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
    lat = np.array([r.latency for r in reqs if not math.isnan(r.t_done)]) * 1e3
    if lat.size == 0:
        return {"count": 0}
    span = max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs)
    return {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "qps": float(lat.size / span) if span > 0 else 0.0,
            "mean_batch": float(np.mean([r.batch_size for r in reqs]))}


class CudaBackend(Backend):
    """The real backend: the C ABI for the scan, torch for buffers, streams and events.

    Every dispatch allocates its batch buffers through torch; with large databases
    run the process with torch's stream-ordered allocator
    (PYTORCH_CUDA_ALLOC_CONF=backend:cudaMallocAsync), whose releases do not
    synchronise the device as the caching allocator's do under memory pressure."""

    def __init__(self, device: int = 0):
        import torch

        import paper_2606_11536_gb300 as g
        self.torch, self.g = torch, g
        self.device = torch.device("cuda", device)

    def setup_db(self, name, params, raw, layout):
        try:
            db = self.g.pir_setup_db(params, raw, layout=layout)
        except self.g.PirError as e:
            if e.status == 3:
                raise AdmissionError("%s: %s" % (name, e)) from e
            raise
        return db, self.g.pir_db_bytes(db)

    def free_db(self, handle):
        self.g.pir_free_db(handle)

    def new_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def dispatch(self, handle, params, queries, stream):
        torch = self.torch
        B = len(queries)
        qwords = params.D1 * 2 * params.L * params.n
        rwords = params.D2 * 2 * params.L * params.n
        with torch.cuda.stream(stream):
            qbuf = torch.empty(B * qwords, dtype=torch.int32, device=self.device)
            for b, q in enumerate(queries):  # gather: one device-to-device copy per request
                qbuf[b * qwords:(b + 1) * qwords].copy_(q, non_blocking=True)
            rbuf = torch.empty(B * rwords, dtype=torch.int32, device=self.device)
            self.g.pir_answer(handle, qbuf, B, rbuf, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev, (qbuf, rbuf)

    def done(self, event) -> bool:
        return event.query()

    def response(self, bufs, b: int, B: int):
        rbuf = bufs[1]
        per = rbuf.numel() // B
        return rbuf[b * per:(b + 1) * per].clone()
