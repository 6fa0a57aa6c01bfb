"""Pins for the oracle's DB encoding, first-dimension folding and toy BFV client:
pure-Python brute force on tiny rings, the schoolbook definition of folding, the
decryption invariant (decrypting the answer returns exactly the requested record),
the paper's worked overflow example, and a Freivalds check that catches a planted
error."""
import numpy as np
import pytest

from golden.read import paper_values
import synth


def py_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for s in range(n):
        for t in range(n):
            k = s + t
            if k < n:
                out[k] = (out[k] + a[s] * b[t]) % q
            else:
                out[k - n] = (out[k - n] - a[s] * b[t]) % q
    return out


def py_coeffs(raw, log2p, n, poly):
    big = int.from_bytes(bytes(raw), "little")
    mask = (1 << log2p) - 1
    return [(big >> ((poly * n + t) * log2p)) & mask for t in range(n)]


@pytest.mark.parametrize("log2p", [4, 8, 12, 16, 13])
def test_unpack_matches_bigint(orc, log2p):
    n, npolys = 16, 5
    raw = synth.raw_db(3, n * npolys * log2p // 8)
    for poly in range(npolys):
        assert [int(v) for v in orc.unpack_poly(raw, log2p, n, poly)] == py_coeffs(raw, log2p, n, poly)
    if log2p == 16:
        u16 = raw.view("<u2").reshape(npolys, n)
        assert np.array_equal(orc.unpack_poly(raw, 16, n, 3), u16[3].astype(np.uint32))


def tiny_instance(orc, n=8, log2p=4, D1=3, D2=2, B=2, seed=9):
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    q = synth.uniform_residues(seed, synth.STREAM_UNIFORM, B * D1 * 2, n, P.qs).reshape(B, D1, 2, 2, n)
    return P, raw, q


def test_answer_brute_force_pure_python(orc):
    P, raw, Q = tiny_instance(orc)
    n, D1, D2, B = P.n, P.D1, P.D2, Q.shape[0]
    got = orc.answer(P, raw, Q)
    for b in range(B):
        for c in range(D2):
            for comp in range(2):
                for j, q in enumerate(P.qs):
                    acc = [0] * n
                    for i in range(D1):
                        d = py_coeffs(raw, P.log2p, n, i * D2 + c)
                        pr = py_negacyclic(d, [int(v) for v in Q[b, i, comp, j]], q)
                        acc = [(x + y) % q for x, y in zip(acc, pr)]
                    assert [int(v) for v in got[b, c, comp, j]] == acc


@pytest.mark.parametrize("n,log2p,D1,D2,B", [(16, 5, 4, 3, 3), (64, 8, 5, 4, 2), (256, 12, 3, 5, 1)])
def test_answer_ntt_route_matches_schoolbook_definition(orc, n, log2p, D1, D2, B):
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(n, synth.raw_db_bytes(n, log2p, D1, D2))
    Q = synth.uniform_residues(n, synth.STREAM_UNIFORM, B * D1 * 2, n, P.qs).reshape(B, D1, 2, 2, n)
    assert np.array_equal(orc.answer(P, raw, Q, nthreads=2), orc.answer_schoolbook(P, raw, Q))
    # column subsets come out identical to the full answer
    full = orc.answer(P, raw, Q)
    cols = np.array([D2 - 1, 0], dtype=np.uint32)
    assert np.array_equal(orc.answer(P, raw, Q, cols=cols), full[:, cols])


def test_encode_then_answer_encoded(orc):
    P, raw, Q = tiny_instance(orc, n=32, log2p=6, D1=4, D2=3, B=2)
    cols = [2, 0]
    ids = np.array([i * P.D2 + c for c in cols for i in range(P.D1)], dtype=np.uint64)
    dbhat = orc.encode_polys(P, raw, ids).reshape(len(cols), P.D1, P.L, P.n)
    for t, pid in enumerate(ids[:3]):
        for j, (q, psi) in enumerate(zip(P.qs, P.psis)):
            d = orc.unpack_poly(raw, P.log2p, P.n, int(pid))
            assert np.array_equal(dbhat.reshape(-1, P.L, P.n)[t, j], orc.ntt_definition(d, q, psi))
    qhat = orc.ntt_fwd_rns(P, Q)
    got = orc.answer_encoded(P, dbhat, qhat)
    assert np.array_equal(got, orc.answer(P, raw, Q, cols=np.array(cols, dtype=np.uint32)))


def client_draws(P, seed, count):
    s = synth.ternary_secret(seed, P.n)
    a = synth.uniform_residues(seed, synth.STREAM_A, count, P.n, P.qs)
    e = synth.gaussian_error(seed, count * P.n).reshape(count, P.n)
    return s, a, e


def test_bfv_roundtrip_and_noise_is_e(orc):
    P = orc.make_params(2048, 12, 1, 1, 2)
    s, a, e = client_draws(P, 21, 3)
    rng = np.random.default_rng(1)
    for t in range(3):
        m = rng.integers(0, 1 << P.log2p, size=P.n).astype(np.uint32)
        ct = orc.bfv_encrypt(P, s, a[t], e[t], m)
        assert np.array_equal(orc.bfv_decrypt(P, s, ct), m)
        assert np.array_equal(orc.bfv_noise(P, s, ct, m), e[t].astype(np.int64))
    pv = paper_values()
    assert np.abs(e).max() <= pv["error_bound"]


def test_paper_overflow_example(orc):
    """App. A.4: (3/8)p + (3/8)p decrypts to -(1/4)p and, taken relative to Delta *
    (-(1/4)p), the phase carries one extra -1 on top of the added errors."""
    pv = paper_values()
    P = orc.make_params(4096, 16, 1, 1, 2)
    p = 1 << P.log2p
    q, delta = orc.modulus_info(P)
    m1 = int(pv["overflow_m1_over_p"] * p)
    s, a, e = client_draws(P, 33, 2)
    m = np.full(P.n, m1, dtype=np.uint32)
    ct1 = orc.bfv_encrypt(P, s, a[0], e[0], m)
    ct2 = orc.bfv_encrypt(P, s, a[1], e[1], m)
    ctsum = np.empty_like(ct1)
    for j, qj in enumerate(P.qs):
        ctsum[:, j] = ((ct1[:, j].astype(np.uint64) + ct2[:, j].astype(np.uint64)) % np.uint64(qj)).astype(np.uint32)
    target = int(pv["overflow_sum_over_p"] * p)  # -(1/4) p
    assert np.array_equal(orc.bfv_decrypt(P, s, ctsum), np.full(P.n, target % p, dtype=np.uint32))
    phi = orc.bfv_phase(P, s, ctsum)
    for t in range(0, P.n, 97):
        resid = (phi[t] - delta * target) % q
        resid = resid - q if resid > q // 2 else resid
        assert resid == int(e[0, t]) + int(e[1, t]) + pv["overflow_extra_error"]


def test_decryption_invariant_tiny_config(orc):
    """The tiny configuration end to end: n = 2048, p = 2^12, 16 x 16 DB from seed 0;
    every response column decrypts to exactly DB[i*][c]."""
    n, log2p, D1, D2 = 2048, 12, 16, 16
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(0, synth.raw_db_bytes(n, log2p, D1, D2))
    assert raw.nbytes == 768 * 1024
    idx = int(synth.query_indices(1, 1, D1, D2)[0])
    i_star, c_star = divmod(idx, D2)
    s, a, e = client_draws(P, 1, D1)
    Q = orc.encrypt_query(P, s, a, e, i_star)[None]
    R = orc.answer(P, raw, Q)
    q, delta = orc.modulus_info(P)
    worst = 0
    for c in range(D2):
        want = orc.unpack_poly(raw, log2p, n, i_star * D2 + c)
        assert np.array_equal(orc.bfv_decrypt(P, s, R[0, c]), want), c
        worst = max(worst, int(np.abs(orc.bfv_noise(P, s, R[0, c], want)).max()))
    assert worst < delta // 2
    # the exact answer agrees with the schoolbook definition on this configuration too
    cols = np.array([c_star], dtype=np.uint32)
    assert np.array_equal(orc.answer(P, raw, Q, cols=cols)[:, 0], R[:, c_star])


def test_freivalds_accepts_correct_and_catches_planted_error(orc):
    n, log2p, D1, D2, B = 64, 8, 6, 5, 2
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(4, synth.raw_db_bytes(n, log2p, D1, D2))
    Q = synth.uniform_residues(4, synth.STREAM_UNIFORM, B * D1 * 2, n, P.qs).reshape(B, D1, 2, 2, n)
    R = orc.answer(P, raw, Q)
    r = synth.freivalds_vector(8, P.qs, D2)
    assert orc.freivalds(P, raw, Q, R, r) == 0
    bad = R.copy()
    bad[1, 3, 0, 1, 17] = (int(bad[1, 3, 0, 1, 17]) + 1) % P.qs[1]
    assert orc.freivalds(P, raw, Q, bad, r) > 0
