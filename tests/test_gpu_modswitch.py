"""GPU parity of modulus switching fused into the inverse NTT (Sec. 4.3; App. D.5):
ntt_inv_modswitch against the oracle's inverse NTT followed by its switch, bit for
bit, for every ring size and L = 1..4, on random residues and on coefficients built
as t Q' + r around the rounding boundary; and pir_answer with PIR_ANSWER_MODSWITCH
on the fused batch-1 path, the batched path, the limb layout, K-chunking, host
buffers and a captured graph, including decryption of every switched column."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, encrypted_queries, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


def switch_gpu(p, polys):
    count = polys.shape[0]
    out = empty_u32(count * p.n)
    g.ntt_inv_modswitch(p, to_dev(polys), out)
    return from_dev(out, (count, p.n))


@pytest.mark.parametrize("n", [2048, 4096, 8192])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_random_residues(orc, n, L):
    p = g.pir_make_params(n, 16, 1, 1, L)
    P = orc.make_params(n, 16, 1, 1, L)
    assert [p.q[j] for j in range(L)] == P.qs
    count = 5
    a = synth.uniform_residues(n + L, synth.STREAM_UNIFORM, count, n, P.qs).reshape(count, L, n)
    want = orc.modswitch(P, orc.ntt_inv_rns(P, a.reshape(count * L, n)).reshape(count, L, n))
    assert np.array_equal(switch_gpu(p, a), want)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_values_at_the_rounding_boundary(orc, L):
    """Coefficients x = t Q' + r with r at 0, (Q'-1)/2, (Q'+1)/2, Q'-1 and random,
    given to the kernel in NTT form; the result is t or t + 1 by construction."""
    n = 2048
    p = g.pir_make_params(n, 16, 1, 1, L)
    P = orc.make_params(n, 16, 1, 1, L)
    q0 = P.qs[0]
    Qd = 1
    for qj in P.qs[1:]:
        Qd *= qj
    half = (Qd - 1) // 2
    rng = np.random.default_rng(L)
    xs, want = [], []
    for k in range(2 * n):
        t = [0, 1, q0 - 1, int(rng.integers(0, q0))][k % 4]
        r = [0, half, half + 1, Qd - 1, int(rng.integers(0, 1 << 62)) % Qd][k % 5]
        xs.append(t * Qd + r)
        want.append((t + (1 if r > half else 0)) % q0)
    coef = np.array([[x % qj for x in xs] for qj in P.qs], dtype=np.uint32)  # [L][2n]
    coef = coef.reshape(L, 2, n).transpose(1, 0, 2).copy()  # [2][L][n]
    hat = orc.ntt_fwd_rns(P, coef.reshape(2 * L, n)).reshape(2, L, n)
    got = switch_gpu(p, hat).reshape(-1)
    assert [int(v) for v in got] == want


def test_arguments(orc):
    p = g.pir_make_params(2048, 16, 1, 1, 2)
    buf = empty_u32(4 * 2 * 2048)
    with pytest.raises(g.PirError) as ei:  # output inside the input
        g.ntt_inv_modswitch(p, buf, buf[2048:], count=2)
    assert ei.value.status == 1
    g.ntt_inv_modswitch(p, buf, empty_u32(4), count=0)  # nothing to do


def instance(orc, n, log2p, D1, D2, seed, layout=0):
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    return p, P, raw, g.pir_setup_db(p, raw, layout=layout)


def answer_switched(db, P, Q, B, **kw):
    rd = empty_u32(B * P.D2 * 2 * P.n)
    g.pir_answer_ex(db, to_dev(Q), B, rd, flags=g.PIR_ANSWER_MODSWITCH, **kw)
    out = from_dev(rd, (B, P.D2, 2, P.n))
    g.pir_check_device()
    return out


@pytest.mark.parametrize("B,layout,kw", [
    (1, 0, {}),                 # fused batch-1 path (TMA scan writes the full-modulus responses to scratch)
    (1, 0, {"k_chunk": 12}),    # fused, K-chunked
    (1, 0, {"tile": 3}),        # batch 1 on the GEMV and the transposes
    (3, 0, {}),                 # batched
    (5, 0, {"k_chunk": 16}),    # batched, K-chunked
    (3, 1, {}),                 # limb layout
])
def test_answer_switched_matches_oracle(orc, B, layout, kw):
    p, P, raw, db = instance(orc, 4096, 16, 64, 20, seed=70 + B, layout=layout)  # limb rows: D1 % 32 == 0
    try:
        Q = random_queries(P, B, 71 + B)
        want = orc.modswitch(P, orc.answer(P, raw, Q))
        assert np.array_equal(answer_switched(db, P, Q, B, **kw), want)
    finally:
        g.pir_free_db(db)


def test_switched_answer_decrypts(orc):
    p, P, raw, db = instance(orc, 2048, 12, 16, 16, seed=0)
    try:
        Q, s, targets = encrypted_queries(orc, P, 2, 1)
        S = answer_switched(db, P, Q, 2)
        for b, (i_star, _) in enumerate(targets):
            for c in range(P.D2):
                want = orc.unpack_poly(raw, P.log2p, P.n, i_star * P.D2 + c)
                assert np.array_equal(orc.bfv_decrypt_q0(P, s, S[b, c]), want), (b, c)
    finally:
        g.pir_free_db(db)


def test_host_buffers_and_graph(orc):
    p, P, raw, db = instance(orc, 2048, 16, 24, 36, seed=9)
    try:
        B = 2
        Q = random_queries(P, B, 10)
        want = orc.modswitch(P, orc.answer(P, raw, Q))
        host = np.zeros((B, P.D2, 2, P.n), dtype=np.uint32)
        g.pir_answer_ex(db, Q, B, host, flags=g.PIR_ANSWER_MODSWITCH)
        assert np.array_equal(host, want)
        qd, rd = to_dev(Q), empty_u32(B * P.D2 * 2 * P.n)
        gr = g.pir_graph_create(db, qd, B, rd, flags=g.PIR_ANSWER_MODSWITCH)
        try:
            g.pir_graph_launch(gr)
            assert np.array_equal(from_dev(rd, want.shape), want)
        finally:
            g.pir_graph_destroy(gr)
    finally:
        g.pir_free_db(db)
