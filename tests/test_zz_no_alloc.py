"""pir_answer_noalloc, the answer for callers that cannot allocate device memory
while serving (a process that reserved its whole device budget up front, or a
latency-critical path that cannot afford an allocator call): its scratch is the
library's fixed per-GPU array.  Called through the C ABI, its output must equal
pir_answer's (exactly: the path is integer) on two calls in a row, and requests
too large for the array must be refused.

Collected last on purpose (file name), so that a run stopping at the first failure
has already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout,n,log2p,D1,D2,B", [
    (0, 2048, 12, 16, 16, 1),     # the tiny configuration
    (0, 4096, 16, 96, 36, 3),     # ragged shape, 6 query rows
    (0, 2048, 16, 64, 20, 9),     # tiled GEMM rows
    (1, 2048, 16, 64, 20, 8),     # limb layout
])
def test_noalloc_matches_pir_answer_twice(orc, layout, n, log2p, D1, D2, B):
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(500 + B, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    try:
        for call in range(2):
            Q = random_queries(P, B, 600 + 10 * B + call)
            qd = to_dev(Q)
            ref_d = empty_u32(B * D2 * 2 * 2 * n)
            g.pir_answer(db, qd, B, ref_d)
            ref = from_dev(ref_d, (B, D2, 2, 2, n))
            out_d = empty_u32(B * D2 * 2 * 2 * n)
            out_d.fill_(-1)
            g.pir_answer_noalloc(db, qd, B, out_d)
            out = from_dev(out_d, (B, D2, 2, 2, n))
            assert np.array_equal(out, ref), call
        assert np.array_equal(ref, orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


@pytest.mark.parametrize("layout", [0, 1])
def test_noalloc_folds_several_k_chunks(orc, layout):
    """A request whose query scratch does not fit the array at once: n = 4096,
    D1 = 512, B = 8 leave room for 63 folded rows beside the 16 MiB result, so the
    answer runs in K chunks (63 rows with a ragged tail on the plain layout, 32 on
    the limb layout), each accumulated into the result.  Equal to pir_answer on two
    calls in a row, and to the oracle on sampled columns."""
    n, log2p, D1, D2, B = 4096, 16, 512, 32, 8
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(520 + layout, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    try:
        for call in range(2):
            Q = random_queries(P, B, 700 + 10 * layout + call)
            qd = to_dev(Q)
            ref_d = empty_u32(B * D2 * 2 * 2 * n)
            g.pir_answer(db, qd, B, ref_d)
            out_d = empty_u32(B * D2 * 2 * 2 * n)
            out_d.fill_(-1)
            g.pir_answer_noalloc(db, qd, B, out_d)
            out = from_dev(out_d, (B, D2, 2, 2, n))
            assert np.array_equal(out, from_dev(ref_d, (B, D2, 2, 2, n))), call
        cols = [0, 17, D2 - 1]
        want = orc.answer(P, raw, Q, cols=cols)
        assert np.array_equal(out[:, cols], want)
    finally:
        g.pir_free_db(db)


def test_noalloc_refuses_requests_beyond_its_scratch(orc):
    # result alone: L*n*2B*D2 words = 2*4096*8*512*4 bytes = 128 MiB > 64 MiB
    n, log2p, D1, D2, B = 4096, 16, 32, 512, 4
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    db = g.pir_setup_db(p, synth.raw_db(7, synth.raw_db_bytes(n, log2p, D1, D2)))
    try:
        qd = empty_u32(B * D1 * 2 * 2 * n)
        rd = empty_u32(B * D2 * 2 * 2 * n)
        with pytest.raises(g.PirError) as ei:
            g.pir_answer_noalloc(db, qd, B, rd)
        assert ei.value.status == 1  # PIR_ERR_ARG
    finally:
        g.pir_free_db(db)
