"""GPU answer parity through the C ABI: pir_setup_db + pir_answer against the
oracle, element by element, on shapes that span several tiles with ragged tails,
every GEMM tile, K-chunked folding, host buffers, and the full-size 1 GiB
configuration (sampled exact columns, a Freivalds check of the whole output and
decryption of every column)."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, encrypted_queries, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


def instance(orc, n, log2p, D1, D2, seed=5, layout=0):
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    return p, P, raw, db


def run(db, P, Q, B, **kw):
    qd = to_dev(Q)
    rd = empty_u32(B * P.D2 * 2 * P.L * P.n)
    if kw:
        g.pir_answer_ex(db, qd, B, rd, **kw)
    else:
        g.pir_answer(db, qd, B, rd)
    out = from_dev(rd, (B, P.D2, 2, P.L, P.n))
    g.pir_check_device()  # no bounded wait ran out
    return out


def test_tiny_config_decrypts_and_matches(orc):
    p, P, raw, db = instance(orc, 2048, 12, 16, 16, seed=0)
    try:
        Q, s, targets = encrypted_queries(orc, P, 1, 1)
        R = run(db, P, Q, 1)
        assert np.array_equal(R, orc.answer(P, raw, Q))
        i_star, _ = targets[0]
        for c in range(P.D2):
            assert np.array_equal(orc.bfv_decrypt(P, s, R[0, c]), orc.unpack_poly(raw, P.log2p, P.n, i_star * P.D2 + c))
    finally:
        g.pir_free_db(db)


def test_db_encoding_matches_oracle(orc):
    p, P, raw, db = instance(orc, 2048, 16, 24, 12, seed=3)
    try:
        assert g.pir_db_bytes(db) == 4 * 2 * 2048 * 24 * 12
        ids = [0, 1, 11, 12, 100, 24 * 12 - 1]
        ref = orc.encode_polys(P, raw, np.array(ids, dtype=np.uint64))
        for t, pid in enumerate(ids):
            assert np.array_equal(g.pir_db_read_poly(db, pid), ref[t])
    finally:
        g.pir_free_db(db)


# M = 2B crosses every kernel: GEMV with 2/4/8 rows, tiled GEMM with 16/32/64-row tiles
@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 8, 9, 16, 17, 33])
def test_batches_ragged_shapes(orc, B):
    p, P, raw, db = instance(orc, 2048, 16, 40, 20, seed=B)
    try:
        Q = random_queries(P, B, 100 + B)
        R = run(db, P, Q, B)
        assert np.array_equal(R, orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


@pytest.mark.parametrize("B,tiles", [(1, (1, 2, 3, 4, 5, 6, 7, 8)), (2, (2, 3, 7, 8)), (4, (3, 7, 8)), (7, (4, 8))])
def test_small_batches_every_tile(orc, B, tiles):
    p, P, raw, db = instance(orc, 4096, 16, 50, 44, seed=60 + B)
    try:
        Q = random_queries(P, B, 61 + B)
        ref = orc.answer(P, raw, Q)
        for tile in tiles:
            assert np.array_equal(run(db, P, Q, B, tile=tile), ref), tile
        if 2 * B <= 8:  # the TMA scan takes at most 8 query rows
            assert np.array_equal(run(db, P, Q, B, tile=7, k_chunk=13), ref)
    finally:
        g.pir_free_db(db)


def test_every_tile_and_k_chunk(orc):
    p, P, raw, db = instance(orc, 2048, 16, 37, 132, seed=9)
    try:
        B = 3
        Q = random_queries(P, B, 11)
        ref = orc.answer(P, raw, Q)
        for tile in range(3, g.pir_gemm_tiles(0) + 1):  # M = 6: tiles 1, 2 hold 2 and 4 rows only
            assert np.array_equal(run(db, P, Q, B, tile=tile), ref), tile
        for k_chunk in (1, 5, 16, 36, 37, 100):
            assert np.array_equal(run(db, P, Q, B, k_chunk=k_chunk), ref), k_chunk
        assert np.array_equal(run(db, P, Q, B, k_chunk=7, tile=6), ref)
    finally:
        g.pir_free_db(db)


def test_ring_8192_and_extreme_values(orc):
    p, P, raw, db = instance(orc, 8192, 16, 8, 8, seed=21)
    try:
        B = 2
        Q = random_queries(P, B, 5)
        for j, q in enumerate(P.qs):  # every query residue q - 1: largest products
            Q[1, :, :, j, :] = q - 1
        assert np.array_equal(run(db, P, Q, B), orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


def test_host_buffers_equal_device_buffers(orc):
    p, P, raw, db = instance(orc, 4096, 16, 16, 8, seed=2)
    try:
        B = 2
        Q = random_queries(P, B, 8)
        Rh = np.empty((B, P.D2, 2, P.L, P.n), dtype=np.uint32)
        g.pir_answer(db, Q, B, Rh)
        assert np.array_equal(Rh, run(db, P, Q, B))
        assert np.array_equal(Rh, orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


def test_errors_on_gpu(orc):
    p, P, raw, db = instance(orc, 2048, 12, 16, 16, seed=0)
    q = empty_u32(16 * 2 * 2 * 2048)
    r = empty_u32(16 * 2 * 2 * 2048)
    with pytest.raises(g.PirError) as ei:
        g.pir_answer(db, q, 0, r)
    assert ei.value.status == 1
    with pytest.raises(g.PirError) as ei:
        g.pir_answer_ex(db, q, 1, r, tile=99)
    assert ei.value.status == 1
    g.pir_free_db(db)
    with pytest.raises(g.PirError) as ei:
        g.pir_answer(db, q, 1, r)  # freed handle
    assert ei.value.status == 6


def test_full_size_1gib_config(orc):
    """n = 4096, p = 2^16, D1 x D2 = 512 x 256 (1 GiB raw, 4 GiB resident), B = 1 real
    encrypted query in the launch configuration the benchmark times: sampled
    columns exact, the whole output by Freivalds, every column decrypts."""
    n, log2p, D1, D2 = 4096, 16, 512, 256
    p, P, raw, db = instance(orc, n, log2p, D1, D2, seed=0)
    try:
        Q, s, targets = encrypted_queries(orc, P, 1, 1)
        R = run(db, P, Q, 1)
        cols = np.array([0, 17, targets[0][1], D2 - 1], dtype=np.uint32)
        assert np.array_equal(R[:, cols], orc.answer(P, raw, Q, cols=cols))
        r = synth.freivalds_vector(3, P.qs, D2)
        assert orc.freivalds(P, raw, Q, R, r) == 0
        i_star = targets[0][0]
        for c in range(D2):
            assert np.array_equal(orc.bfv_decrypt(P, s, R[0, c]), orc.unpack_poly(raw, log2p, n, i_star * D2 + c)), c
    finally:
        g.pir_free_db(db)


# --- the INT8 limb path (u8 x u8 -> s32 tensor-pipe products) ----------------

@pytest.mark.parametrize("B", [1, 3, 8, 9, 16, 17, 32, 40])
def test_limb_path_matches_oracle(orc, B):
    p, P, raw, db = instance(orc, 2048, 16, 64, 20, seed=30 + B, layout=1)
    try:
        Q = random_queries(P, B, 200 + B)
        assert np.array_equal(run(db, P, Q, B), orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


def test_limb_tiles_chunks_and_encoding(orc):
    p, P, raw, db = instance(orc, 2048, 16, 96, 36, seed=44, layout=1)
    try:
        ids = [0, 35, 36, 95 * 36 + 35]
        ref = orc.encode_polys(P, raw, np.array(ids, dtype=np.uint64))
        for t, pid in enumerate(ids):
            assert np.array_equal(g.pir_db_read_poly(db, pid), ref[t])
        B = 32  # Mp = 64: every tile shape fits
        Q = random_queries(P, B, 9)
        for j, q in enumerate(P.qs):  # one query of all-maximal residues
            Q[0, :, :, j, :] = q - 1
        ref = orc.answer(P, raw, Q)
        for tile in (1, 2, 3):
            assert np.array_equal(run(db, P, Q, B, tile=tile), ref), tile
        for k_chunk in (32, 64, 40):
            assert np.array_equal(run(db, P, Q, B, k_chunk=k_chunk), ref), k_chunk
    finally:
        g.pir_free_db(db)


def test_limb_full_size_1gib_batch8(orc):
    """The 1 GiB configuration on the limb path at B = 8: sampled columns exact,
    the whole output by Freivalds."""
    n, log2p, D1, D2 = 4096, 16, 512, 256
    p, P, raw, db = instance(orc, n, log2p, D1, D2, seed=0, layout=1)
    try:
        B = 8
        Q = random_queries(P, B, 77)
        R = run(db, P, Q, B)
        cols = np.array([0, 101, D2 - 1], dtype=np.uint32)
        assert np.array_equal(R[:, cols], orc.answer(P, raw, Q, cols=cols))
        assert orc.freivalds(P, raw, Q, R, synth.freivalds_vector(4, P.qs, D2)) == 0
    finally:
        g.pir_free_db(db)


@pytest.mark.parametrize("D1,B,k_chunk", [(99, 1, 26), (99, 1, 0), (120, 1, 0), (118, 1, 0), (64, 3, 0)])
def test_host_buffers_pipelined_upload_and_odd_chunks(orc, D1, B, k_chunk):
    """Host-buffer answers whose upload is split into pieces on a copy stream (queries
    of 8 MiB and more): batch 1 keeps one scan pass with the forward NTT following the
    pieces (D1 = 120, 118: equal and ragged pieces), an odd D1 takes the unfused path,
    batch 3 scans K-chunk by K-chunk; and an odd D1 with an even chunk size."""
    n = 8192 if D1 >= 100 else 4096
    p, P, raw, db = instance(orc, n, 16, D1, 8, seed=D1 + B)
    try:
        Q = random_queries(P, B, 77 + D1)
        ref = orc.answer(P, raw, Q)
        host = np.zeros(ref.shape, dtype=np.uint32)
        g.pir_answer_ex(db, Q, B, host, k_chunk=k_chunk)
        assert np.array_equal(host, ref)
        assert np.array_equal(run(db, P, Q, B, k_chunk=k_chunk), ref)
    finally:
        g.pir_free_db(db)


@pytest.mark.parametrize("layout,B,flags", [(0, 17, 0), (0, 24, 4), (2, 32, 0), (2, 20, 4)])
def test_host_buffers_sub_batch_pipeline(orc, layout, B, flags):
    """Host batches of 16 and more queries (8 MiB and more) run as sub-batches of at
    least 8 queries (ragged at B = 17, 20): uploads, answers and downloads overlap
    on three streams; equal to the oracle, with and without modulus switching."""
    p, P, raw, db = instance(orc, 2048, 16, 64, 32, seed=B + layout, layout=layout)
    try:
        Q = random_queries(P, B, 300 + B)
        ref = orc.answer(P, raw, Q)
        if flags & g.PIR_ANSWER_MODSWITCH:
            ref = orc.modswitch(P, ref)
        host = np.zeros(ref.shape, dtype=np.uint32)
        g.pir_answer_ex(db, Q, B, host, flags=flags)
        assert np.array_equal(host, ref)
    finally:
        g.pir_free_db(db)


def test_check_inputs_refuses_non_canonical_residues(orc):
    """PIR_ANSWER_CHECK_INPUTS: canonical queries answer as without the check (device
    and host buffers); one residue equal to its prime is refused with PIR_ERR_ARG,
    whichever prime's row it sits in."""
    n, log2p, D1, D2, B = 2048, 16, 32, 16, 3
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(31, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw)
    try:
        Q = random_queries(P, B, 32)
        want = orc.answer(P, raw, Q)
        rd = empty_u32(want.size)
        g.pir_answer_ex(db, to_dev(Q), B, rd, flags=g.PIR_ANSWER_CHECK_INPUTS)
        assert np.array_equal(from_dev(rd, want.shape), want)
        rh = np.empty(want.size, dtype=np.uint32)
        g.pir_answer_ex(db, np.ascontiguousarray(Q).reshape(-1), B, rh, flags=g.PIR_ANSWER_CHECK_INPUTS)
        assert np.array_equal(rh.reshape(want.shape), want)
        for (b, i, comp, j, t) in ((0, 0, 0, 0, 0), (B - 1, D1 - 1, 1, 1, n - 1), (1, 7, 0, 1, 5)):
            bad = Q.copy()
            bad[b, i, comp, j, t] = P.qs[j]
            with pytest.raises(g.PirError) as ei:
                g.pir_answer_ex(db, to_dev(bad), B, rd, flags=g.PIR_ANSWER_CHECK_INPUTS)
            assert ei.value.status == 1
        g.pir_answer_ex(db, to_dev(bad), B, rd)  # without the check the call is not refused
    finally:
        g.pir_free_db(db)
