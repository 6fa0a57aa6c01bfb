"""GPU parity of the bf16 tensor-core path (PIR_LAYOUT_TENSOR: signed base-256 digits
of every residue, tcgen05.mma with f32 accumulators in tensor memory) through the C
ABI, bit for bit against the oracle: DB encoding, answers for batches that cross
the query-row tiles (1..64 queries) on shapes with ragged column tiles, K-chunks
(explicit, rounded to 64-row blocks, and the automatic 1024-row bound), all-(q-1)
queries, modulus switching, host buffers, streamed pieces, a captured graph, the
no-allocation entry point, the autotuner, and the full 1 GiB configuration at
batch 32 (sampled columns exact, the whole output by Freivalds)."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu
TENSOR = 2


def instance(orc, n, D1, D2, seed, log2p=16):
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    return p, P, raw, g.pir_setup_db(p, raw, layout=TENSOR)


def run(db, P, Q, B, msw=False, **kw):
    rd = empty_u32(B * P.D2 * 2 * (1 if msw else P.L) * P.n)
    if msw:
        kw["flags"] = kw.get("flags", 0) | g.PIR_ANSWER_MODSWITCH
    g.pir_answer_ex(db, to_dev(Q), B, rd, **kw)
    out = from_dev(rd, (B, P.D2, 2, P.n) if msw else (B, P.D2, 2, P.L, P.n))
    g.pir_check_device()  # no bounded wait ran out
    return out


def test_db_encoding_and_resident_bytes(orc):
    p, P, raw, db = instance(orc, 2048, 64, 96, seed=90)
    try:
        assert g.pir_db_bytes(db) == 8 * 2 * 2048 * 64 * 96
        ids = [0, 1, 95, 96, 63 * 96, 64 * 96 - 1, 1000]
        ref = orc.encode_polys(P, raw, np.array(ids, dtype=np.uint64))
        for t, pid in enumerate(ids):
            assert np.array_equal(g.pir_db_read_poly(db, pid), ref[t])
    finally:
        g.pir_free_db(db)


# M = 2B query rows pad to 8; B > 32 takes a second query-row tile
@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 8, 9, 16, 17, 32, 33, 40])
def test_batches_match_oracle(orc, B):
    p, P, raw, db = instance(orc, 2048, 128, 96, seed=91 + B)
    try:
        Q = random_queries(P, B, 92 + B)
        assert np.array_equal(run(db, P, Q, B), orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


def test_wide_columns_and_batch_64(orc):
    """D2 = 512: sixteen 32-column tiles per CTA at small batches; batch 64 = two
    full query-row tiles."""
    p, P, raw, db = instance(orc, 2048, 64, 512, seed=93)
    try:
        for B in (2, 64):
            Q = random_queries(P, B, 94 + B)
            cols = np.array([0, 31, 32, 255, 256, 511], dtype=np.uint32)
            R = run(db, P, Q, B)
            assert np.array_equal(R[:, cols], orc.answer(P, raw, Q, cols=cols)), B
            assert orc.freivalds(P, raw, Q, R, synth.freivalds_vector(5, P.qs, P.D2)) == 0
    finally:
        g.pir_free_db(db)


def test_k_chunks_and_the_1024_row_bound(orc):
    """D1 = 2112 (> 1024): the f32-exactness bound splits D1 into chunks of at most
    1024 rows on its own; explicit chunks round down to 64-row blocks."""
    p, P, raw, db = instance(orc, 2048, 2112, 32, seed=95)
    try:
        B = 3
        Q = random_queries(P, B, 96)
        ref = orc.answer(P, raw, Q)
        assert np.array_equal(run(db, P, Q, B), ref)
        for k_chunk in (64, 100, 640, 1024, 4096):
            assert np.array_equal(run(db, P, Q, B, k_chunk=k_chunk), ref), k_chunk
    finally:
        g.pir_free_db(db)


def test_extreme_residues_and_n8192(orc):
    p, P, raw, db = instance(orc, 8192, 64, 32, seed=97)
    try:
        B = 4
        Q = random_queries(P, B, 98)
        for j, q in enumerate(P.qs):  # every residue of query 1 is q - 1
            Q[1, :, :, j, :] = q - 1
        Q[2] = 0
        assert np.array_equal(run(db, P, Q, B), orc.answer(P, raw, Q))
    finally:
        g.pir_free_db(db)


def test_modswitch_host_buffers_and_streamed(orc):
    p, P, raw, db = instance(orc, 4096, 192, 64, seed=99)
    try:
        B = 6
        Q = random_queries(P, B, 100)
        ref = orc.answer(P, raw, Q)
        assert np.array_equal(run(db, P, Q, B, msw=True), orc.modswitch(P, ref))
        host = np.zeros(ref.shape, dtype=np.uint32)
        g.pir_answer_ex(db, Q, B, host)
        assert np.array_equal(host, ref)
        ses = g.pir_answer_begin(db, B, 128)
        for i0, kc in ((0, 64), (64, 128)):
            g.pir_answer_chunk(ses, np.ascontiguousarray(Q[:, i0:i0 + kc]), i0, kc)
        out = np.zeros(ref.shape, dtype=np.uint32)
        g.pir_answer_end(ses, out)
        assert np.array_equal(out, ref)
        ses = g.pir_answer_begin(db, B, 128)
        with pytest.raises(g.PirError) as ei:  # pieces are whole 64-row blocks
            g.pir_answer_chunk(ses, np.ascontiguousarray(Q[:, 0:32]), 0, 32)
        assert ei.value.status == 1
        g.pir_answer_abort(ses)
    finally:
        g.pir_free_db(db)


def test_graph_noalloc_and_autotune(orc):
    p, P, raw, db = instance(orc, 2048, 128, 32, seed=101)
    try:
        B = 8
        Q = random_queries(P, B, 102)
        ref = orc.answer(P, raw, Q)
        qd, rd = to_dev(Q), empty_u32(ref.size)
        graph = g.pir_graph_create(db, qd, B, rd)
        try:
            g.pir_graph_launch(graph)
            assert np.array_equal(from_dev(rd, ref.shape), ref)
        finally:
            g.pir_graph_destroy(graph)
        rd2 = empty_u32(ref.size)
        g.pir_answer_noalloc(db, qd, B, rd2)
        assert np.array_equal(from_dev(rd2, ref.shape), ref)
        best = g.pir_autotune(db, B)
        assert best["tile"] == 1 and best["k_chunk"] in (0, 64)
        assert np.array_equal(run(db, P, Q, B, **best), ref)
        with pytest.raises(g.PirError) as ei:
            run(db, P, Q, B, tile=2)
        assert ei.value.status == 1
    finally:
        g.pir_free_db(db)


def test_unsupported_shapes():
    for D1, D2 in ((96, 32), (64, 48)):
        p = g.pir_make_params(2048, 16, D1, D2, 2)
        raw = np.zeros(synth.raw_db_bytes(2048, 16, D1, D2), dtype=np.uint8)
        with pytest.raises(g.PirError) as ei:
            g.pir_setup_db(p, raw, layout=TENSOR)
        assert ei.value.status == 7, (D1, D2)


def test_full_size_1gib_batch32(orc):
    """The 1 GiB configuration (n = 4096, 512 x 256; 8 GiB resident in this layout)
    at B = 32, in the launch configuration the benchmark times."""
    n, D1, D2 = 4096, 512, 256
    p, P, raw, db = instance(orc, n, D1, D2, seed=0)
    try:
        B = 32
        Q = random_queries(P, B, 103)
        R = run(db, P, Q, B)
        cols = np.array([0, 77, D2 - 1], dtype=np.uint32)
        assert np.array_equal(R[:3][:, cols], orc.answer(P, raw, Q[:3], cols=cols))
        assert np.array_equal(R[-1:][:, cols], orc.answer(P, raw, Q[-1:], cols=cols))
        assert orc.freivalds(P, raw, Q, R, synth.freivalds_vector(6, P.qs, D2)) == 0
    finally:
        g.pir_free_db(db)


# --- exactness at the f32 boundary -------------------------------------------
#
# A residue x < 2^30 becomes signed base-256 digits d_0..d_2 in [-128, 127] and
# d_3 in [0, 64].  0x7F7F80 has digits (-128, -128, -128, 1), so over a 1024-row
# K-chunk every (-128) x (-128) digit-pair sum is exactly 1024 * 2^14 = 2^24, the
# largest integer whose every partial sum f32 must carry without rounding.
# 0x7F7F7F has digits (127, 127, 127, 0).  With p = 2^23 both values are
# plaintext coefficients, so a DB of constant polynomials v_i holds v_i in every
# NTT slot, and so does a query of constant polynomials w_i.  The response to every
# query row and column is then the constant polynomial sum_i v_i w_i mod q_j: a
# closed form, checked on every output, besides the oracle on sampled columns.

V_MIN, V_MAX = 0x7F7F80, 0x7F7F7F


def digits(x):
    out = []
    for _ in range(3):
        d = x & 255
        x >>= 8
        if d >= 128:
            d -= 256
            x += 1
        out.append(d)
    return out + [x]


def constant_db(n, log2p, D1, D2, values):
    """Raw DB whose polynomial (i, c) is the constant values[i] (log2p-bit LE stream)."""
    bpp = n * log2p // 8
    raw = np.zeros((D1, D2, bpp), dtype=np.uint8)
    v = np.asarray(values, dtype=np.uint64)
    for k in range(3):
        raw[:, :, k] = ((v >> np.uint64(8 * k)) & np.uint64(255)).astype(np.uint8)[:, None]
    return raw.reshape(-1)


@pytest.mark.parametrize("case", ["all_minus_128", "alternating_extremes"])
def test_digit_sums_of_exactly_2_to_24(orc, case):
    assert digits(V_MIN) == [-128, -128, -128, 1] and digits(V_MAX) == [127, 127, 127, 0]
    n, log2p, D1, D2, B = 2048, 23, 2048, 64, 8
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    assert p.qs == P.qs and all(q > V_MIN for q in p.qs)
    if case == "all_minus_128":
        v = [V_MIN] * D1
        w = [V_MIN] * D1
    else:  # digit products alternate between +2^14 and -128 * 127 along K
        v = [V_MIN] * D1
        w = [V_MIN if i % 2 == 0 else V_MAX for i in range(D1)]
    raw = constant_db(n, log2p, D1, D2, v)
    Q = np.zeros((B, D1, 2, 2, n), dtype=np.uint32)
    Q[..., 0] = np.asarray(w, dtype=np.uint32)[None, :, None, None]
    db = g.pir_setup_db(p, raw, layout=TENSOR)
    try:
        R = run(db, P, Q, B)
    finally:
        g.pir_free_db(db)
    for j, q in enumerate(P.qs):
        want = sum(a * b for a, b in zip(v, w)) % q
        assert np.all(R[:, :, :, j, 0] == want), j
        assert not R[:, :, :, j, 1:].any(), j
    cols = np.array([0, D2 - 1], dtype=np.uint32)
    assert np.array_equal(R[[0, B - 1]][:, cols], orc.answer(P, raw, Q[[0, B - 1]], cols=cols))


def test_full_size_16gib_batches_32_and_128(orc):
    """The 16 GiB configuration (n = 4096, 4096 x 512; 128 GiB resident in this
    layout) at B = 32 and B = 128, in the launch configuration the benchmark times
    (automatic K-chunks of 1024 rows), on sampled (query, column) outputs the
    oracle computes one by one."""
    import torch
    from test_gpu_fullsize import device_queries, host_query, oracle_columns, setup_on_device
    n, log2p, D1, D2 = 4096, 16, 4096, 512
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    db = setup_on_device(p, 0, layout=TENSOR)
    try:
        assert g.pir_db_bytes(db) == 128 << 30
        for B in (32, 128):
            seed = 140 + B
            qd = device_queries(P, B, seed)
            rd = torch.empty(B * D2 * 2 * 2 * n, dtype=torch.int32, device="cuda")
            g.pir_answer(db, qd, B, rd)
            R = rd.view(B, D2, 2, 2, n)
            for b, cs in ((0, [3, 300]), (B // 2 + 1, [31, 32]), (B - 1, [511, 64])):
                got = R[b, cs].cpu().numpy().view(np.uint32)
                assert np.array_equal(got[None], oracle_columns(orc, P, 0, cs, host_query(P, b, seed))), (B, b)
            g.pir_check_device()
            del qd, rd, R
            torch.cuda.empty_cache()
    finally:
        g.pir_free_db(db)
        torch.cuda.empty_cache()


@pytest.mark.parametrize("B", [1, 4, 32, 40, 64])
def test_one_sm_and_two_sm_forms_agree_with_the_oracle(orc, B):
    """The 1-SM GEMM (tile 1), the CTA-pair GEMM (tile 2: one tcgen05 MMA over two
    SMs, M = 256), the 1-SM GEMM in clusters of two (tile 3) and the CTA pair with
    tensor-map loads (tile 5, where the query rows allow it) against the oracle, on D2 = 192 (three column-tile pairs), query
    rows that leave a ragged second 256-row tile at B = 40 and 64, and two K-chunks."""
    p, P, raw, db = instance(orc, 2048, 256, 192, seed=130 + B)
    try:
        Q = random_queries(P, B, 131 + B)
        cols = np.array([0, 63, 64, 191], dtype=np.uint32)
        want = orc.answer(P, raw, Q, cols=cols)
        Ntot = 4 * ((2 * B + 7) // 8 * 8)
        tma_ok = Ntot <= 256 or Ntot % 256 == 0  # the tensor-map pair form's one box size
        for tile in (1, 2, 3) + ((5,) if tma_ok else ()):
            for kc in (0, 128):
                R = run(db, P, Q, B, tile=tile, k_chunk=kc)
                assert np.array_equal(R[:, cols], want), (tile, kc)
        R1, R2 = run(db, P, Q, B, tile=1), run(db, P, Q, B, tile=2)
        assert np.array_equal(R1, R2)
        assert np.array_equal(R1, run(db, P, Q, B, tile=3))
        if tma_ok:
            assert np.array_equal(R1, run(db, P, Q, B, tile=5))
        else:
            with pytest.raises(g.PirError) as ei:  # a ragged second query tile: refused
                run(db, P, Q, B, tile=5)
            assert ei.value.status == 1
    finally:
        g.pir_free_db(db)


@pytest.mark.parametrize("B", [1, 8, 32, 40, 64])
def test_cluster_multicast_forms_agree_with_the_oracle(orc, B):
    """The 1-SM GEMM in clusters of 2 and 4 CTAs (tiles 3 and 4), each CTA loading a
    share of every stage's query digits and multicasting it to the cluster: D2 = 256
    (eight 32-column tiles, so groups of 2 and 4 units of one slot), small batches
    with several column tiles per unit, the ragged second 256-row query tile at
    B = 40 and 64, and two K-chunks; equal to the oracle and to tile 1 everywhere."""
    p, P, raw, db = instance(orc, 2048, 128, 256, seed=150 + B)
    try:
        Q = random_queries(P, B, 151 + B)
        cols = np.array([0, 31, 32, 127, 128, 255], dtype=np.uint32)
        want = orc.answer(P, raw, Q, cols=cols)
        R1 = run(db, P, Q, B, tile=1)
        assert np.array_equal(R1[:, cols], want)
        for tile in (3, 4):
            for kc in (0, 64):
                R = run(db, P, Q, B, tile=tile, k_chunk=kc)
                assert np.array_equal(R[:, cols], want), (tile, kc)
                assert np.array_equal(R, R1), (tile, kc)
        g.pir_check_device()
    finally:
        g.pir_free_db(db)


def test_cluster_forms_refuse_column_counts_they_cannot_split(orc):
    p, P, raw, db = instance(orc, 2048, 64, 96, seed=160)
    try:
        Q = random_queries(P, 2, 161)
        for tile in (3, 4, 5):
            with pytest.raises(g.PirError) as ei:
                run(db, P, Q, 2, tile=tile)
            assert ei.value.status == 1, tile
    finally:
        g.pir_free_db(db)
