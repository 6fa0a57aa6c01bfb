"""Serving on the GPU: several resident databases, requests arriving while others
run, coalesced into batches on several streams.  Each response must be exactly the
response of the same query answered alone (and the oracle's), and admission must
refuse a database the memory budget cannot hold."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
from paper_2606_11536_gb300 import serving
import synth

pytestmark = pytest.mark.gpu

SHAPES = {  # name -> (n, log2p, D1, D2, layout)
    "small_n2048": (2048, 16, 32, 16, 0),
    "small_n4096": (4096, 16, 16, 8, 0),
    "limb_n2048": (2048, 16, 64, 12, 1),
}


@pytest.mark.parametrize("graphs", [False, True])
def test_mixed_requests_equal_their_answers_alone(orc, graphs):
    """With graphs, each batch runs as a captured, autotuned answer padded with zero
    queries to its power-of-two bucket; the answers must not change."""
    be = serving.CudaBackend(graphs=graphs, max_batch=4)
    srv = serving.Server(be, streams=3, max_batch=4, keep_responses=True, batch_timeout=60.0)
    pools, raws, P = {}, {}, {}
    for k, (name, (n, log2p, D1, D2, layout)) in enumerate(SHAPES.items()):
        p = g.pir_make_params(n, log2p, D1, D2, 2)
        P[name] = orc.make_params(n, log2p, D1, D2, 2)
        raws[name] = synth.raw_db(40 + k, synth.raw_db_bytes(n, log2p, D1, D2))
        srv.admit(name, p, raws[name], layout=layout)
        Q = random_queries(P[name], 6, 70 + k)
        pools[name] = [to_dev(Q[b]) for b in range(6)]
    # a burst: 40 requests over ~2 ms, random databases
    rng = np.random.default_rng(9)
    names = list(SHAPES)
    arrivals = []
    for rid in range(40):
        db = names[rng.integers(len(names))]
        arrivals.append(serving.Request(rid, db, (db, int(rng.integers(6))), float(rid) * 5e-5))
    for r in arrivals:
        r.query = pools[r.db][r.query[1]]
    done = srv.run(arrivals)
    assert len(done) == 40 and all(np.isfinite(r.t_done) for r in done)
    assert max(r.batch_size for r in done) > 1  # the mix really was batched
    for r in done:
        n, log2p, D1, D2, layout = SHAPES[r.db]
        alone = empty_u32(D2 * 2 * 2 * n)
        g.pir_answer(srv.dbs[r.db]["handle"], r.query, 1, alone)
        assert np.array_equal(from_dev(r.response), from_dev(alone)), (r.rid, r.db, r.batch_size)
    # and one of them against the oracle
    r = done[0]
    Qh = from_dev(r.query).reshape(1, SHAPES[r.db][2], 2, 2, SHAPES[r.db][0])
    assert np.array_equal(from_dev(r.response).reshape(1, SHAPES[r.db][3], 2, 2, SHAPES[r.db][0]),
                          orc.answer(P[r.db], raws[r.db], Qh))
    g.pir_check_device()
    st = serving.latency_stats(done)
    assert st["count"] == 40 and st["p99_ms"] >= st["p50_ms"] > 0 and st["failed"] == 0
    if graphs:
        assert be.graph_launches == len({(r.t_dispatch, r.db) for r in done})  # every batch ran as a graph
    for name in names:
        srv.evict(name)


def test_admission_refuses_what_the_budget_cannot_hold():
    be = serving.CudaBackend()
    n, log2p, D1, D2 = 2048, 16, 32, 16
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    one = 4 * 2 * n * D1 * D2
    srv = serving.Server(be, streams=1, memory_budget=2 * one + one // 2)
    raw = synth.raw_db(3, synth.raw_db_bytes(n, log2p, D1, D2))
    srv.admit("a", p, raw)
    srv.admit("b", p, raw)
    with pytest.raises(serving.AdmissionError):
        srv.admit("c", p, raw)
    assert len(srv.dbs) == 2
    srv.evict("a")
    srv.admit("c", p, raw)
    srv.evict("b")
    srv.evict("c")
