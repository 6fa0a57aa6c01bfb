"""GPU parity of the streamed answer (pir_answer_begin / chunk / end; Sec. 4.4,
stream-wise buffering): the queries are given in pieces along D1, ragged and of
several sizes, from host and device memory, on the plain and the limb layout, with
and without modulus switching; every result equals the oracle's answer bit for bit.
Then the argument rules (order, range, limb blocks, finished and aborted sessions)
and host batches above 4 GiB, which pir_answer_ex streams in pieces (plain and tensor layouts)."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


def instance(orc, n, D1, D2, seed, layout=0):
    p = g.pir_make_params(n, 16, D1, D2, 2)
    P = orc.make_params(n, 16, D1, D2, 2)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, 16, D1, D2))
    return p, P, raw, g.pir_setup_db(p, raw, layout=layout)


def streamed(db, P, Q, B, pieces, kc_max, host, flags=0, tile=0):
    ses = g.pir_answer_begin(db, B, kc_max, flags=flags, tile=tile)
    i0 = 0
    for kc in pieces:
        part = np.ascontiguousarray(Q[:, i0:i0 + kc])
        g.pir_answer_chunk(ses, part if host else to_dev(part), i0, kc)
        i0 += kc
    shape = (B, P.D2, 2, P.n) if flags & g.PIR_ANSWER_MODSWITCH else (B, P.D2, 2, P.L, P.n)
    if host:
        out = np.zeros(shape, dtype=np.uint32)
        g.pir_answer_end(ses, out)
        return out
    rd = empty_u32(np.prod(shape))
    g.pir_answer_end(ses, rd)
    return from_dev(rd, shape)


@pytest.mark.parametrize("B,pieces,kc_max,host", [
    (1, (40,), 40, False),           # one piece
    (1, (7, 13, 20), 20, True),      # ragged, host staging ping-pong
    (3, (1, 1, 38), 38, False),
    (3, (16, 16, 8), 16, True),
    (9, (11, 29), 64, True),          # the tiled GEMM, kc_max above D1
])
def test_streamed_answer_plain(orc, B, pieces, kc_max, host):
    p, P, raw, db = instance(orc, 2048, 40, 20, seed=70 + B)
    try:
        Q = random_queries(P, B, 71 + B)
        assert np.array_equal(streamed(db, P, Q, B, pieces, kc_max, host), orc.answer(P, raw, Q))
        g.pir_check_device()
    finally:
        g.pir_free_db(db)


@pytest.mark.parametrize("host", [False, True])
def test_streamed_answer_modswitch_and_tile(orc, host):
    p, P, raw, db = instance(orc, 4096, 24, 12, seed=80)
    try:
        B = 2
        Q = random_queries(P, B, 81)
        want = orc.modswitch(P, orc.answer(P, raw, Q))
        assert np.array_equal(streamed(db, P, Q, B, (10, 10, 4), 10, host, flags=g.PIR_ANSWER_MODSWITCH), want)
        assert np.array_equal(streamed(db, P, Q, B, (5, 19), 19, host, tile=8), orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


def test_streamed_answer_limb(orc):
    p, P, raw, db = instance(orc, 2048, 96, 20, seed=82, layout=1)
    try:
        B = 5
        Q = random_queries(P, B, 83)
        ref = orc.answer(P, raw, Q)
        assert np.array_equal(streamed(db, P, Q, B, (32, 64), 64, False), ref)
        assert np.array_equal(streamed(db, P, Q, B, (32, 32, 32), 40, True), ref)  # kc_max rounds to 32
    finally:
        g.pir_free_db(db)


def status_of(fn, *a, **kw):
    with pytest.raises(g.PirError) as ei:
        fn(*a, **kw)
    return ei.value.status


def test_streamed_answer_arguments(orc):
    p, P, raw, db = instance(orc, 2048, 16, 8, seed=84)
    pl, PL, rawl, dbl = instance(orc, 2048, 64, 8, seed=85, layout=1)
    try:
        B = 1
        Q = random_queries(P, B, 85)
        assert status_of(g.pir_answer_begin, db, 0, 4) == 1
        assert status_of(g.pir_answer_begin, db, B, 0) == 1
        assert status_of(g.pir_answer_begin, db, B, 4, flags=g.PIR_ANSWER_TEST_STALL) == 1
        assert status_of(g.pir_answer_begin, db, B, 4, tile=99) == 1
        ses = g.pir_answer_begin(db, B, 8)
        assert status_of(g.pir_answer_chunk, ses, Q[:, 4:8].copy(), 4, 4) == 1      # not the next piece
        assert status_of(g.pir_answer_chunk, ses, Q[:, 0:9].copy(), 0, 9) == 1      # above kc_max
        assert status_of(g.pir_answer_chunk, ses, Q[:, 0:0].copy(), 0, 0) == 1      # empty piece
        g.pir_answer_chunk(ses, Q[:, 0:8].copy(), 0, 8)
        with pytest.raises(ValueError):  # the binding: 8 ciphertexts given, 9 declared
            g.pir_answer_chunk(ses, Q[:, 8:16].copy(), 8, 9)
        past = np.zeros((B, 9, 2, P.L, P.n), dtype=np.uint32)
        assert status_of(g.pir_answer_chunk, ses, past, 8, 9) == 1                  # past D1
        rd = empty_u32(P.D2 * 2 * P.L * P.n)
        assert status_of(g.pir_answer_end, ses, rd) == 1                             # half of D1: released
        assert status_of(g.pir_answer_chunk, ses, Q[:, 8:16].copy(), 8, 8) == 6
        ses = g.pir_answer_begin(db, B, 8)
        g.pir_answer_chunk(ses, Q[:, 0:8].copy(), 0, 8)
        g.pir_answer_abort(ses)
        assert status_of(g.pir_answer_abort, ses) == 6
        ses = g.pir_answer_begin(dbl, B, 64)
        Ql = random_queries(PL, B, 86)
        assert status_of(g.pir_answer_chunk, ses, Ql[:, 0:16].copy(), 0, 16) == 1  # limb pieces: 32-row blocks
        g.pir_answer_abort(ses)
        # the whole answer still works after the refused calls
        assert np.array_equal(streamed(db, P, Q, B, (8, 8), 8, False), orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)
        g.pir_free_db(dbl)


def test_host_batch_above_4gib_streams(orc):
    """B x D1 x 32 KiB = 4.06 GiB of host queries: pir_answer_ex streams them in
    pieces of at most 1 GiB.  Equal to the device-buffer answer (itself pinned to the
    oracle above); query 0 checked against the oracle on sampled columns."""
    import torch
    n, D1, D2, B = 2048, 16640, 4, 8
    p, P, raw, db = instance(orc, n, D1, D2, seed=86)
    try:
        qd = torch.empty(B * D1 * 2 * 2 * n, dtype=torch.int32, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(87)
        for j, q in enumerate(P.qs):  # residues below each prime, prime-major rows
            view = qd.view(B * D1 * 2, 2, n)[:, j]
            view.copy_(torch.randint(0, q, view.shape, device="cuda", generator=gen, dtype=torch.int64).to(torch.int32))
        Qh = from_dev(qd, (B, D1, 2, 2, n))
        assert Qh.nbytes > (4 << 30)
        rd = empty_u32(B * D2 * 2 * 2 * n)
        g.pir_answer_ex(db, qd, B, rd)
        want = from_dev(rd, (B, D2, 2, 2, n))
        host = np.zeros_like(want)
        g.pir_answer_ex(db, Qh, B, host)
        assert np.array_equal(host, want)
        cols = np.array([0, 3], dtype=np.uint32)
        assert np.array_equal(host[:1, cols], orc.answer(P, raw, Qh[:1], cols=cols))
    finally:
        g.pir_free_db(db)


def test_host_batch_above_4gib_streams_tensor_layout(orc):
    """The same on the tensor layout, whose streamed pieces are sized from the
    available device memory (whole 64-row blocks, at most 1024 rows): 4.1 GiB of host
    queries, equal to the device-buffer answer and to the oracle on sampled columns."""
    import torch
    n, D1, D2, B = 2048, 16640, 32, 8
    p = g.pir_make_params(n, 16, D1, D2, 2)
    P = orc.make_params(n, 16, D1, D2, 2)
    raw = synth.raw_db(88, synth.raw_db_bytes(n, 16, D1, D2))
    db = g.pir_setup_db(p, raw, layout=2)
    try:
        qd = torch.empty(B * D1 * 2 * 2 * n, dtype=torch.int32, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(89)
        for j, q in enumerate(P.qs):
            view = qd.view(B * D1 * 2, 2, n)[:, j]
            view.copy_(torch.randint(0, q, view.shape, device="cuda", generator=gen, dtype=torch.int64).to(torch.int32))
        Qh = from_dev(qd, (B, D1, 2, 2, n))
        assert Qh.nbytes > (4 << 30)
        rd = empty_u32(B * D2 * 2 * 2 * n)
        g.pir_answer_ex(db, qd, B, rd)
        want = from_dev(rd, (B, D2, 2, 2, n))
        host = np.zeros_like(want)
        g.pir_answer_ex(db, Qh, B, host)
        assert np.array_equal(host, want)
        cols = np.array([0, 31], dtype=np.uint32)
        assert np.array_equal(host[-1:, cols], orc.answer(P, raw, Qh[-1:], cols=cols))
    finally:
        g.pir_free_db(db)
