"""GPU parity of the folding of the remaining dimensions (Sec. 3.2, 3.6; App. D.3)
through the C ABI: pir_fold against the oracle's fold, bit for bit, for L = 1..3,
n = 2048 and 4096, depths 1..4 and several digit counts; pir_answer_folded against
the oracle's first-dimension answer folded the same way (batch 1 and batched, with
modulus switching, host buffers); one-record decryption end to end; argument checks."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, encrypted_queries, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,levels,ell", [(2048, 1, 3, 3), (2048, 2, 1, 4), (2048, 2, 4, 6), (4096, 2, 3, 4),
                                            (2048, 3, 2, 4)])
def test_fold_matches_oracle(orc, n, L, levels, ell):
    p = g.pir_make_params(n, 16, 1, 1, L)
    P = orc.make_params(n, 16, 1, 1, L)
    B, count = 2, 1 << levels
    cts = synth.uniform_residues(n + levels, synth.STREAM_UNIFORM, B * count * 2, n, P.qs).reshape(B, count, 2, L, n)
    rgsw = synth.uniform_residues(ell, synth.STREAM_KEY_A, B * levels * 2 * ell * 2, n, P.qs).reshape(
        B, levels, 2 * ell, 2, L, n)
    out = empty_u32(B * 2 * L * n)
    g.pir_fold(p, to_dev(cts), B, levels, ell, to_dev(rgsw), out)
    got = from_dev(out, (B, 2, L, n))
    for b in range(B):
        assert np.array_equal(got[b], orc.fold(P, cts[b], levels, rgsw[b], ell)), b


def db_instance(orc, n, log2p, D1, D2, seed):
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    return p, P, raw, g.pir_setup_db(p, raw)


@pytest.mark.parametrize("B,flags", [(1, 0), (3, 0), (2, 4)])
def test_answer_folded_matches_oracle(orc, B, flags):
    ell = 4
    p, P, raw, db = db_instance(orc, 2048, 16, 40, 16, seed=B + 50)
    try:
        levels = 4
        Q = random_queries(P, B, 51 + B)
        rgsw = synth.uniform_residues(7, synth.STREAM_KEY_A, B * levels * 2 * ell * 2, P.n, P.qs).reshape(
            B, levels, 2 * ell, 2, P.L, P.n)
        R = orc.answer(P, raw, Q)
        want = np.stack([orc.fold(P, R[b], levels, rgsw[b], ell) for b in range(B)])
        if flags & g.PIR_ANSWER_MODSWITCH:
            want = orc.modswitch(P, want)
        rd = empty_u32(want.size)
        g.pir_answer_folded(db, to_dev(Q), B, ell, to_dev(rgsw), rd, flags=flags)
        assert np.array_equal(from_dev(rd, want.shape), want)
        g.pir_check_device()
        host = np.zeros(want.shape, dtype=np.uint32)
        g.pir_answer_folded(db, Q, B, ell, rgsw, host, flags=flags)
        assert np.array_equal(host, want)
    finally:
        g.pir_free_db(db)


def test_folded_answer_decrypts_the_record(orc):
    ell = 6
    p, P, raw, db = db_instance(orc, 2048, 12, 16, 16, seed=0)
    try:
        B = 2
        Q, s, targets = encrypted_queries(orc, P, B, 1)
        rgsw = np.stack([orc.rgsw_bits(P, s, [(c >> l) & 1 for l in range(4)], ell, seed=10 + b)
                         for b, (_, c) in enumerate(targets)])
        rd = empty_u32(B * 2 * P.L * P.n)
        g.pir_answer_folded(db, to_dev(Q), B, ell, to_dev(rgsw), rd)
        out = from_dev(rd, (B, 2, P.L, P.n))
        for b, (i_star, c_star) in enumerate(targets):
            want = orc.unpack_poly(raw, P.log2p, P.n, i_star * P.D2 + c_star)
            assert np.array_equal(orc.bfv_decrypt(P, s, out[b]), want), b
    finally:
        g.pir_free_db(db)


def test_arguments(orc):
    p, P, raw, db = db_instance(orc, 2048, 16, 8, 12, seed=4)  # D2 = 12: not a power of two
    try:
        Q = to_dev(np.zeros((1, 8, 2, 2, P.n), dtype=np.uint32))
        G = to_dev(np.zeros((1, 4, 8, 2, 2, P.n), dtype=np.uint32))
        with pytest.raises(g.PirError) as ei:
            g.pir_answer_folded(db, Q, 1, 4, G, empty_u32(2 * 2 * P.n))
        assert ei.value.status == 1
        with pytest.raises(g.PirError) as ei:  # one digit of 60 bits
            g.pir_fold(p, Q, 1, 1, 1, G, empty_u32(2 * 2 * P.n))
        assert ei.value.status == 1
    finally:
        g.pir_free_db(db)
