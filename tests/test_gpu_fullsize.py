"""Full-size parity for the 16 GiB (n = 4096, 4096 x 512) and 32 GiB (n = 8192,
8192 x 256) databases and the serving configuration's 1 GiB n = 2048 (512 x 512)
and 8 GiB (2048 x 512) ones, in the launch configuration bench.py times (default tile
and K-chunk choice), on outputs the oracle computes one by one: sampled
(query, column) responses exact, and for batch 1 a real encrypted query whose
sampled columns decrypt to the requested records.  The databases and large query
batches are generated on the device from the same counter-based streams the
oracle regenerates on the host."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, encrypted_queries, from_dev, to_dev
import synth

pytestmark = pytest.mark.gpu


def oracle_columns(orc, P, db_seed, cols, Qb):
    """Oracle responses [1][len(cols)][2][L][n] of one query Qb [1][D1][2][L][n] for
    the given columns, from the raw slabs of just those DB polynomials."""
    bpp = P.n * P.log2p // 8
    compact = np.concatenate([synth.raw_db_slab(db_seed, (i * P.D2 + c) * bpp, bpp) for c in cols for i in range(P.D1)])
    Pc = orc.make_params(P.n, P.log2p, len(cols) * P.D1, 1, P.L)
    dbhat = orc.encode_polys(Pc, compact, np.arange(len(cols) * P.D1, dtype=np.uint64))
    dbhat = dbhat.reshape(len(cols), P.D1, P.L, P.n)
    return orc.answer_encoded(P, dbhat, orc.ntt_fwd_rns(P, Qb))


def setup_on_device(p, seed, layout=0):
    import torch
    raw = synth.raw_db_torch(seed, p.D1 * p.D2 * p.n * p.log2p // 8, device="cuda")
    db = g.pir_setup_db(p, raw, layout=layout)
    del raw
    torch.cuda.empty_cache()
    return db


def device_queries(P, B, seed):
    return synth.uniform_residues_torch(seed, synth.STREAM_UNIFORM, B * P.D1 * 2, P.n, P.qs, device="cuda").view(-1)


def host_query(P, b, seed):
    return synth.uniform_residues(seed, synth.STREAM_UNIFORM, P.D1 * 2, P.n, P.qs, start=b * P.D1 * 2).reshape(
        1, P.D1, 2, P.L, P.n)


def test_16gib_database_batches_1_8_32_128(orc):
    import torch
    n, log2p, D1, D2 = 4096, 16, 4096, 512
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    db = setup_on_device(p, 0)
    try:
        assert g.pir_db_bytes(db) == 64 << 30
        # batch 1: a real encrypted query, the fused scan path
        Q, s, targets = encrypted_queries(orc, P, 1, 1)
        rd = empty_u32(D2 * 2 * 2 * n)
        g.pir_answer(db, to_dev(Q), 1, rd)
        R = from_dev(rd, (1, D2, 2, 2, n))
        i_star, c_star = targets[0]
        cols = sorted({0, c_star, 333, D2 - 1})
        bpp = n * log2p // 8
        for c in cols:
            want = orc.unpack_poly(synth.raw_db_slab(0, (i_star * D2 + c) * bpp, bpp), log2p, n, 0)
            assert np.array_equal(orc.bfv_decrypt(P, s, R[0, c]), want), c
        exact = oracle_columns(orc, P, 0, [c_star, 77], Q)
        assert np.array_equal(R[:, [c_star, 77]], exact)
        # batches 8, 32, 128 of uniform query ciphertexts
        for B in (8, 32, 128):
            seed = 40 + B
            qd = device_queries(P, B, seed)
            rd = torch.empty(B * D2 * 2 * 2 * n, dtype=torch.int32, device="cuda")
            g.pir_answer(db, qd, B, rd)
            R = rd.view(B, D2, 2, 2, n)
            for b, cs in ((0, [5, 400]), (B - 1, [511, 128])):
                got = R[b, cs].cpu().numpy().view(np.uint32)
                assert np.array_equal(got[None], oracle_columns(orc, P, 0, cs, host_query(P, b, seed))), (B, b)
            del qd, rd, R
            torch.cuda.empty_cache()
        g.pir_check_device()
    finally:
        g.pir_free_db(db)


def test_32gib_database_batch64_plain_and_limb(orc):
    import torch
    n, log2p, D1, D2, B, seed = 8192, 16, 8192, 256, 64, 91
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    samples = ((3, [0, 200]), (B - 1, [255, 17]))
    expect = {b: oracle_columns(orc, P, 1, cs, host_query(P, b, seed)) for b, cs in samples}
    for layout in (0, 1):
        db = setup_on_device(p, 1, layout=layout)
        try:
            assert g.pir_db_bytes(db) == 128 << 30
            qd = device_queries(P, B, seed)
            rd = torch.empty(B * D2 * 2 * 2 * n, dtype=torch.int32, device="cuda")
            g.pir_answer(db, qd, B, rd)
            R = rd.view(B, D2, 2, 2, n)
            for b, cs in samples:
                got = R[b, cs].cpu().numpy().view(np.uint32)
                assert np.array_equal(got[None], expect[b]), (layout, b)
            g.pir_check_device()
            del qd, rd, R
        finally:
            g.pir_free_db(db)
            torch.cuda.empty_cache()


@pytest.mark.parametrize("n,D1,D2,B,seed", [(2048, 512, 512, 8, 21), (4096, 2048, 512, 32, 22)])
def test_serving_configuration_databases(orc, n, D1, D2, B, seed):
    """The two database shapes only the serving configuration uses: 1 GiB at n = 2048
    (512 x 512) and the 8 GiB fourth database at n = 4096 (2048 x 512), each at a
    serving-sized batch, on sampled (query, column) outputs against the oracle."""
    import torch
    log2p = 16
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    db = setup_on_device(p, seed)
    try:
        qd = device_queries(P, B, seed + 100)
        rd = torch.empty(B * D2 * 2 * 2 * n, dtype=torch.int32, device="cuda")
        g.pir_answer(db, qd, B, rd)
        R = rd.view(B, D2, 2, 2, n)
        for b, cs in ((0, [0, D2 - 1]), (B - 1, [D2 // 2, 7])):
            got = R[b, cs].cpu().numpy().view(np.uint32)
            assert np.array_equal(got[None], oracle_columns(orc, P, seed, cs, host_query(P, b, seed + 100))), b
        g.pir_check_device()
    finally:
        g.pir_free_db(db)
        torch.cuda.empty_cache()
