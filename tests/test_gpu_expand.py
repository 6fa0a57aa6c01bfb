"""GPU parity of server-side query expansion (Sec. 3.5; App. C.2; App. D.3) through
the C ABI: pir_expand against the oracle's expansion, bit for bit, for L = 1..4,
several depths and digit counts, full and partial outputs; pir_answer_packed
against the oracle's answer to the expanded queries on the batch-1 and batched
paths, the limb layout, modulus switching and host buffers; decryption of every
column for a real packed one-hot query; and the argument checks."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, to_dev
import synth

pytestmark = pytest.mark.gpu


def keys_and_packed(orc, P, levels, ell, B, seed):
    s = synth.ternary_secret(seed, P.n)
    keys = orc.expansion_keys(P, s, levels, ell, seed=seed)
    packed = synth.uniform_residues(seed, synth.STREAM_UNIFORM, 2 * B, P.n, P.qs).reshape(B, 2, P.L, P.n)
    return s, keys, packed


@pytest.mark.parametrize("n,L,levels,ell", [
    (2048, 1, 3, 2), (2048, 2, 3, 4), (2048, 2, 4, 6), (4096, 2, 5, 4), (2048, 3, 4, 4), (2048, 4, 2, 5),
    (8192, 2, 2, 3),
])
def test_expand_matches_oracle(orc, n, L, levels, ell):
    p = g.pir_make_params(n, 16, 1, 1, L)
    P = orc.make_params(n, 16, 1, 1, L)
    B = 2
    _, keys, packed = keys_and_packed(orc, P, levels, ell, B, seed=n + L + levels)
    ex = g.pir_expander_create(p, levels, ell, keys)
    try:
        for count in sorted({1 << levels, max(1, (1 << levels) - 3)}):
            out = empty_u32(B * count * 2 * L * n)
            g.pir_expand(ex, to_dev(packed), B, count, out)
            got = from_dev(out, (B, count, 2, L, n))
            for b in range(B):
                want = orc.expand(P, packed[b], levels, ell, keys, count)
                assert np.array_equal(got[b], want), (b, count)
    finally:
        g.pir_expander_free(ex)


def packed_instance(orc, n, log2p, D1, D2, L, ell, seed, layout=0):
    p = g.pir_make_params(n, log2p, D1, D2, L)
    P = orc.make_params(n, log2p, D1, D2, L)
    levels = (D1 - 1).bit_length()
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    return p, P, levels, raw, db


@pytest.mark.parametrize("B,layout,flags", [(1, 0, 0), (3, 0, 0), (2, 1, 0), (1, 0, 4), (5, 0, 4)])
def test_answer_packed_matches_oracle(orc, B, layout, flags):
    ell = 4
    p, P, levels, raw, db = packed_instance(orc, 2048, 16, 64, 20, 2, ell, seed=90 + B, layout=layout)
    _, keys, packed = keys_and_packed(orc, P, levels, ell, B, seed=91 + B)
    ex = g.pir_expander_create(p, levels, ell, keys)
    try:
        Q = np.stack([orc.expand(P, packed[b], levels, ell, keys, P.D1) for b in range(B)])
        want = orc.answer(P, raw, Q)
        L = 1 if flags & g.PIR_ANSWER_MODSWITCH else P.L
        if flags & g.PIR_ANSWER_MODSWITCH:
            want = orc.modswitch(P, want)
        rd = empty_u32(B * P.D2 * 2 * L * P.n)
        g.pir_answer_packed(db, ex, to_dev(packed), B, rd, flags=flags)
        assert np.array_equal(from_dev(rd, want.shape), want)
        g.pir_check_device()
        host = np.zeros(want.shape, dtype=np.uint32)
        g.pir_answer_packed(db, ex, packed, B, host, flags=flags)
        assert np.array_equal(host, want)
    finally:
        g.pir_expander_free(ex)
        g.pir_free_db(db)


@pytest.mark.parametrize("L,log2p,D1,D2,ell", [(2, 12, 16, 16, 6), (3, 16, 32, 8, 4)])
def test_packed_one_hot_query_decrypts(orc, L, log2p, D1, D2, ell):
    p, P, levels, raw, db = packed_instance(orc, 2048, log2p, D1, D2, L, ell, seed=3)
    s = synth.ternary_secret(7, P.n)
    keys = orc.expansion_keys(P, s, levels, ell, seed=7)
    ex = g.pir_expander_create(p, levels, ell, keys)
    try:
        B = 2
        idx = synth.query_indices(7, B, D1, D2)
        packed = np.stack([
            orc.encrypt_packed_query(P, s, synth.uniform_residues(7, synth.STREAM_A, 1, P.n, P.qs, start=b)[0],
                                     synth.gaussian_error(7, P.n, start=b * P.n), int(idx[b]) // D2)
            for b in range(B)])
        rd = empty_u32(B * D2 * 2 * L * P.n)
        g.pir_answer_packed(db, ex, to_dev(packed), B, rd)
        R = from_dev(rd, (B, D2, 2, L, P.n))
        for b in range(B):
            i_star = int(idx[b]) // D2
            for c in range(D2):
                want = orc.unpack_poly(raw, log2p, P.n, i_star * D2 + c)
                assert np.array_equal(orc.bfv_decrypt(P, s, R[b, c]), want), (b, c)
    finally:
        g.pir_expander_free(ex)
        g.pir_free_db(db)


def test_arguments(orc):
    p, P, levels, raw, db = packed_instance(orc, 2048, 16, 16, 4, 2, 4, seed=5)
    p4 = g.pir_make_params(4096, 16, 1, 1, 2)
    P4 = orc.make_params(4096, 16, 1, 1, 2)
    s = synth.ternary_secret(1, P.n)
    shallow = g.pir_expander_create(p, levels - 1, 4, orc.expansion_keys(P, s, levels - 1, 4, seed=1))
    other = g.pir_expander_create(p4, levels, 4, orc.expansion_keys(P4, synth.ternary_secret(1, 4096), levels, 4, 1))
    try:
        packed = to_dev(np.zeros((1, 2, 2, P.n), dtype=np.uint32))
        rd = empty_u32(P.D2 * 2 * 2 * P.n)
        for ex in (shallow, other):  # too few levels for D1; another ring
            with pytest.raises(g.PirError) as ei:
                g.pir_answer_packed(db, ex, packed, 1, rd)
            assert ei.value.status == 1
        with pytest.raises(g.PirError) as ei:  # more outputs than 2^levels
            g.pir_expand(shallow, packed, 1, 1 << levels, empty_u32((1 << levels) * 2 * 2 * P.n))
        assert ei.value.status == 1
        with pytest.raises(g.PirError) as ei:  # digits wider than 30 bits
            g.pir_expander_create(p, levels, 1, np.zeros((levels, 1, 2, 2, P.n), dtype=np.uint32))
        assert ei.value.status == 1
    finally:
        g.pir_expander_free(shallow)
        g.pir_expander_free(other)
        g.pir_free_db(db)


def _phase_rows(orc, P, s, ct):
    """Phase c_a s + c_b of a ciphertext [2][L][n], one row per prime."""
    out = []
    for j, q in enumerate(P.qs):
        sq = (np.asarray(s, dtype=np.int64) % q).astype(np.uint32)
        out.append((orc.negacyclic_schoolbook(ct[0, j], sq, q).astype(np.uint64) + ct[1, j]) % q)
    return np.stack(out).astype(np.uint32)


def _shift_div(a, C, q):
    """a X^-C in Z_q[X]/(X^n + 1)."""
    a = a.astype(np.int64)
    return np.concatenate([a[C:], (q - a[:C]) % q]).astype(np.uint32) if C else a.astype(np.uint32)


@pytest.mark.parametrize("n,L,levels,ell", [(2048, 1, 3, 3), (2048, 2, 3, 4), (2048, 3, 2, 5)])
def test_expand_phases_with_error_free_keys(orc, n, L, levels, ell):
    """Keys with uniform masks and zero errors add no noise, so whatever digit order a
    key switch uses, expanded ciphertext k must have exactly the phase of SealPIR's
    recursion run on phases: phi <- 2^-levels phi, then per level (g = n/2^j + 1,
    C = 2^j) phi_k + tau_g(phi_k) at k and phi_k X^-C + tau_g(phi_k X^-C) at k + C."""
    p = g.pir_make_params(n, 16, 1, 1, L)
    P = orc.make_params(n, 16, 1, 1, L)
    s = synth.ternary_secret(n + L, n)
    zero_e = np.zeros((ell, n), dtype=np.int8)
    keys = np.stack([orc.ksk_gen(P, s, gal, ell, synth.uniform_residues(lev + 5, synth.STREAM_KEY_A, ell, n, P.qs),
                                 zero_e) for lev, gal in enumerate(orc.expansion_galois(n, levels))])
    packed = synth.uniform_residues(L + 9, synth.STREAM_UNIFORM, 2, n, P.qs).reshape(1, 2, L, n)
    count = 1 << levels
    ex = g.pir_expander_create(p, levels, ell, keys)
    try:
        out = empty_u32(count * 2 * L * n)
        g.pir_expand(ex, to_dev(packed), 1, count, out)
        got = from_dev(out, (count, 2, L, n))
    finally:
        g.pir_expander_free(ex)
    phi = _phase_rows(orc, P, s, packed[0])
    for j, q in enumerate(P.qs):
        cur = [(phi[j].astype(np.uint64) * pow(1 << levels, -1, q) % q).astype(np.uint32)]
        for lev, gal in enumerate(orc.expansion_galois(n, levels)):
            C = 1 << lev
            nxt = [None] * (2 * C)
            for k in range(C):
                sh = _shift_div(cur[k], C, q)
                nxt[k] = ((cur[k].astype(np.uint64) + orc.automorphism(cur[k], q, gal)) % q).astype(np.uint32)
                nxt[k + C] = ((sh.astype(np.uint64) + orc.automorphism(sh, q, gal)) % q).astype(np.uint32)
            cur = nxt
        for k in range(count):
            assert np.array_equal(_phase_rows(orc, P, s, got[k])[j], cur[k]), (j, k)


@pytest.mark.parametrize("B,flags", [(1, 0), (3, 4)])
def test_graph_of_packed_answer(orc, B, flags):
    """pir_graph_create_packed: the expansion and the answer captured once, replayed
    twice on new packed queries in the bound buffer, equal to pir_answer_packed; and
    refused once its expander is freed."""
    ell = 4
    p, P, levels, raw, db = packed_instance(orc, 2048, 16, 64, 20, 2, ell, seed=150 + B)
    _, keys, packed = keys_and_packed(orc, P, levels, ell, B, seed=151 + B)
    ex = g.pir_expander_create(p, levels, ell, keys)
    try:
        Lr = 1 if flags else 2
        pd = to_dev(packed)
        rg = empty_u32(B * 20 * 2 * Lr * 2048)
        graph = g.pir_graph_create_packed(db, ex, pd, B, rg, flags=flags)
        try:
            for rep in range(2):
                newp = synth.uniform_residues(152 + rep, synth.STREAM_UNIFORM, 2 * B, P.n, P.qs).reshape(B, 2, 2, P.n)
                pd.copy_(to_dev(newp))
                g.pir_graph_launch(graph)
                ref = empty_u32(rg.numel())
                g.pir_answer_packed(db, ex, to_dev(newp), B, ref, flags=flags)
                assert np.array_equal(from_dev(rg), from_dev(ref)), rep
        finally:
            g.pir_expander_free(ex)
            with pytest.raises(g.PirError) as ei:
                g.pir_graph_launch(graph)
            assert ei.value.status == 6
            g.pir_graph_destroy(graph)
    finally:
        g.pir_free_db(db)
